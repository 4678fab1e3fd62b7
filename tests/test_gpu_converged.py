"""Converged-run parity and element-wise force parity of the CUDA path with
the FP64 oracle.

Converged runs (Algorithm 2, fixed omega of Sec. 5.2.1; relative
displacement 1e-4, at most 1000 iterations): the oracle's runs are stored in
tests/golden/converged_runs.json by tests/golden/make_converged.py (oracle
only).  Families: Erdos-Renyi n = 2000 (disconnected, unreachable pairs at
(largest d) + 1), random binary tree n = 2047, Delaunay n = 2000, at
classical omega 1.0 / 1.5 / 1.9, with the CG and the direct solver; and eight
graphs of the 4096-graph batched workload through the batched kernel and the
single-graph path.  Bounds: final stress within 1e-4 relative; iteration
counts within 2 % (at least 1), so both runs stop at the cap or both
converge; the outcome of line 6 equal over the first 20 iterations.

Forces, element by element: |F_ic - F_ic^oracle| <= 1e-5 A_ic with
A_ic = sum_j |w_ij (d_ij / r_ij - 1)(x_ic - x_jc)| (oracle.force_row_abs), the
magnitude of the terms the row sums, so that a few wrong rows cannot hide
under a norm over all vertices.  Checked at X^0, along a run (iterations 1,
5 and 20: both sides evaluate F at the GPU's layout), and at a layout the
oracle converged, where F is close to 0 and only the cancellation is left.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "converged_runs.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _iters_close(a, b):
    return abs(a - b) <= max(1, math.ceil(0.02 * b))


def _script():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_converged", os.path.join(HERE, "golden", "make_converged.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


FAMILY_CASES = [(name, om) for name in ("er2000", "tree2047", "delaunay2000") for om in (0.0, 0.5, 0.9)]


@pytest.mark.parametrize("solver", [api.SOLVER_CG, api.SOLVER_DIRECT])
@pytest.mark.parametrize("name,omega", FAMILY_CASES)
def test_converged_family_runs(name, omega, solver):
    g = _golden()
    ref = next(c for c in g["cases"] if c["kind"] == "family" and c["key"] == name and c["omega"] == omega)
    rp, ci = _script().family_graph(name)
    n = len(rp) - 1
    X = synth.initial_layout(n, 2, 0)
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        if solver == api.SOLVER_DIRECT:
            L.factor()
        r = L.run(X, trace=True, omega=omega, tol=g["tol"], max_iter=g["max_iter"], stop=api.STOP_REL_DISP,
                  solver=solver)
    msg = f"{name} omega={omega}: gpu {r.iterations} it f={r.stress}, oracle {ref['iterations']} it f={ref['stress']}"
    assert r.stress == pytest.approx(ref["stress"], rel=1e-4), msg
    assert _iters_close(r.iterations, ref["iterations"]), msg
    assert (r.iterations < g["max_iter"]) == ref["converged"], msg
    k = min(20, len(ref["accept"]), r.iterations)
    assert list(map(bool, r.accepted[:k])) == ref["accept"][:k], msg
    assert np.allclose(r.trace_f[:k + 1], ref["trace_f"][:k + 1], rtol=1e-4, atol=0), msg


def test_batched_sample_matches_oracle():
    g = _golden()
    cases = [c for c in g["cases"] if c["kind"] == "batch"]
    mk = _script()
    graphs = [mk.batch_graph(c["key"]) for c in cases]
    sizes = synth.batch_sizes(mk.BATCH_GRAPHS, seed=0)
    X0 = np.concatenate([synth.initial_layout(int(sizes[c["key"]]), 2, c["key"]) for c in cases])
    opts = dict(omega=0.5, tol=g["tol"], max_iter=g["max_iter"], stop=api.STOP_REL_DISP)
    with api.Batch.from_graphs(graphs, dim=2, disconnected_policy=1) as B:
        X = X0.copy()
        res = B.run(X, **opts)
    off = 0
    for i, c in enumerate(cases):
        n = c["n"]
        with api.Layout(*graphs[i], dim=2, disconnected_policy=1) as L:
            r = L.run(X0[off:off + n].copy(), **opts)
        off += n
        for who, it, f in (("batched", int(res.iterations[i]), float(res.stress[i])),
                           ("single", r.iterations, r.stress)):
            msg = f"graph {c['key']} (n={n}) {who}: {it} it f={f}; oracle {c['iterations']} it f={c['stress']}"
            assert f == pytest.approx(c["stress"], rel=1e-4), msg
            assert _iters_close(it, c["iterations"]), msg


# ---------------------------------------------------------------------------
# forces, element by element
# ---------------------------------------------------------------------------

FORCE_GRAPHS = {
    "grid20": lambda: synth.grid(20, 20),
    "er300": lambda: synth.erdos_renyi(300, 4.0, seed=1),
    "tree383": lambda: synth.random_binary_tree(383, seed=2),
    "delaunay1000": lambda: synth.delaunay(1000, seed=3),
    "rgg2049": lambda: synth.random_geometric(2049, 2, 6.0, seed=5)[:2],
}


def _check_rows(F, X, D, what):
    """|F_ic - F_ic^oracle| <= 1e-5 A_ic for every element."""
    F = np.asarray(F, dtype=np.float64)
    ref = oracle.forces(X, D)
    A = oracle.force_abs(X, D)
    err = np.abs(F - ref)
    ratio = err / np.maximum(A, 1e-300)
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert np.all(err <= 1e-5 * A + 1e-30), (
        f"{what}: worst element {worst} err {err[worst]:.3e} A {A[worst]:.3e} (ratio {ratio[worst]:.3e}); "
        f"rows over the bound: {int(np.sum(np.any(err > 1e-5 * A, axis=1)))}")
    return float(ratio.max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("name", list(FORCE_GRAPHS))
def test_forces_elementwise_along_a_run(name, dim):
    rp, ci = FORCE_GRAPHS[name]()
    n = len(rp) - 1
    st, D = oracle.apsp(rp, ci, policy=1)
    X0 = synth.initial_layout(n, dim, seed=11)
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        _check_rows(L.forces(X0), X0, D, "X0")
        X = X0.copy()
        done = 0
        for k in (1, 5, 20):
            r = L.run(X, omega=0.5, tol=0.0, max_iter=k - done, first_iter=done)
            assert r.iterations == k - done
            done = k
            _check_rows(L.forces(X), X.astype(np.float64), D, f"iteration {k}")


@pytest.mark.parametrize("name", ["grid20", "er300", "tree383", "delaunay1000"])
def test_forces_elementwise_at_converged_layout(name):
    # the oracle's converged layout (relative stress decrease 1e-9), rounded to
    # FP32: F is close to 0 there and every row is a cancellation
    rp, ci = FORCE_GRAPHS[name]()
    n = len(rp) - 1
    st, D = oracle.apsp(rp, ci, policy=1)
    X0 = synth.initial_layout(n, 2, seed=1).astype(np.float64)
    ref = oracle.sor_run(D, X0, omega=0.5, tol=1e-9, stop=oracle.STOP_REL_STRESS, max_iter=1500)
    Xc = ref.X.astype(np.float32)
    F0 = oracle.forces(X0, D)
    Fc = oracle.forces(Xc, D)
    assert np.linalg.norm(Fc) < 1e-2 * np.linalg.norm(F0)  # converged: F is small
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        _check_rows(L.forces(Xc), Xc.astype(np.float64), D, "converged")
