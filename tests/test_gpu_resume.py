"""Checkpoint and resume of a layout run: the state of Algorithm 2 between
iterations is the layout X^k and the iteration index k (the probabilistic
strategy's k-th draw, Sec. 5.2.3).  A run interrupted after k iterations
and resumed from its X^k with first_iter = k must follow the uninterrupted
run: the same omega sequence and acceptance decisions, and the same layout
up to the rounding of the per-vertex atomic sums."""
import numpy as np
import pytest

from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


@pytest.mark.parametrize("solver", [0, 1])
def test_interrupted_run_resumes_exactly(solver):
    rp, ci = synth.delaunay(1500, seed=4)
    n = len(rp) - 1
    X0 = synth.initial_layout(n, 2, seed=4)
    opts = dict(strategy=api.OMEGA_PROB, seed=77, tol=0.0, solver=solver)
    with api.Layout(rp, ci, dim=2) as L:
        if solver == api.SOLVER_DIRECT:
            L.factor()
        Xa = X0.copy()
        ra = L.run(Xa, trace=True, max_iter=40, **opts)
        Xb = X0.copy()
        r1 = L.run(Xb, trace=True, max_iter=15, **opts)
        ckpt = Xb.copy()  # the checkpoint: X^15 (and k = 15)
        Xc = ckpt.copy()
        r2 = L.run(Xc, trace=True, max_iter=25, first_iter=15, **opts)
    assert ra.iterations == 40 and r1.iterations == 15 and r2.iterations == 25
    assert np.array_equal(np.concatenate([r1.omega, r2.omega]), ra.omega)
    assert np.array_equal(np.concatenate([r1.accepted, r2.accepted]), ra.accepted)
    assert r2.stress == pytest.approx(ra.stress, rel=1e-6)
    assert np.linalg.norm(Xc - Xa) <= 1e-5 * np.linalg.norm(Xa)


def test_first_iter_must_not_be_negative():
    rp, ci = synth.grid(5, 5)
    with api.Layout(rp, ci, dim=2) as L:
        with pytest.raises(api.FdError) as e:
            L.run(synth.initial_layout(25, 2, 0), first_iter=-1)
        assert e.value.status == 1
