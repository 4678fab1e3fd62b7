"""The direct solver of Eq. (2-5) through the C ABI, against the FP64 oracle.

fd_factor inverts A' = L^W + (sigma/n) 1 1^T once (FP32 Gauss-Jordan in
128 x 128 blocks); every H step then refines x += A'^-1 r, r -= L^W A'^-1 r
until the same relative residual as CG (cg_tol).

Tolerances:
  rows of A'^-1   1e-4 relative (row norm).  Gauss-Jordan on a positive
                  definite matrix is backward stable, so the forward error is
                  about sqrt(n) kappa eps_32 ~ 45 * 13 * 6e-8 = 4e-5 at
                  n = 2049 with kappa(A') <= 13 on these graphs.
  SOR step / run  as for CG: 1e-4 relative on the layout of one step; final
                  stress 1e-4 relative and iterations within 2 % (at least 1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


def _lengths(rp, ci, seed):
    """Symmetric edge lengths, uniform in [0.5, 2] per unordered edge."""
    rng = np.random.default_rng(seed)
    w = np.empty(len(ci), np.float32)
    lens = {}
    for i in range(len(rp) - 1):
        for e in range(rp[i], rp[i + 1]):
            key = (min(i, ci[e]), max(i, ci[e]))
            lens.setdefault(key, np.float32(rng.uniform(0.5, 2.0)))
            w[e] = lens[key]
    return w


def _D(rp, ci, edge_len=None):
    st, D = oracle.apsp(rp, ci, edge_len=edge_len, policy=1)
    return D


GRAPHS = {
    "k2": (lambda: synth.path(2), 2),
    "grid20": (lambda: synth.grid(20, 20), 2),
    "er300": (lambda: synth.erdos_renyi(300, 4.0, seed=1), 3),
    "tree383": (lambda: synth.random_binary_tree(383, seed=2), 1),
    "delaunay1000": (lambda: synth.delaunay(1000, seed=3), 2),
    "rgg2049": (lambda: synth.random_geometric(2049, 2, 6.0, seed=5)[:2], 2),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_factor_rows_match_oracle(name):
    g, dim = GRAPHS[name]
    rp, ci = g()
    n = len(rp) - 1
    Ai = oracle.shifted_inverse(_D(rp, ci))
    rows = sorted(set([0, n - 1] + list(np.random.default_rng(0).integers(0, n, 6))))
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        L.factor()
        assert L.info()["factored"] == 1
        for r in rows:
            got = L.factor_rows(r, 1)[0]
            assert np.linalg.norm(got - Ai[r]) <= 1e-4 * np.linalg.norm(Ai[r]), r


def test_factor_rows_weighted_graph():
    rp, ci = synth.grid(12, 12)
    ln = _lengths(rp, ci, 3)
    n = len(rp) - 1
    Ai = oracle.shifted_inverse(_D(rp, ci, edge_len=ln.astype(np.float64)))
    with api.Layout(rp, ci, dim=2, edge_len=ln) as L:
        L.factor()
        got = L.factor_rows(0, n)
    assert np.linalg.norm(got - Ai) <= 1e-4 * np.linalg.norm(Ai)


@pytest.mark.parametrize("name,omega", [("grid20", 0.5), ("er300", 0.5), ("tree383", 0.0), ("delaunay1000", 1.0)])
def test_one_sor_step_matches_oracle(name, omega):
    g, dim = GRAPHS[name]
    rp, ci = g()
    n = len(rp) - 1
    D = _D(rp, ci)
    X0 = synth.initial_layout(n, dim, seed=5)
    Xn, fn, acc, _, _ = oracle.sor_step(X0.astype(np.float64), D, omega)
    X = X0.copy()
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        L.factor()
        f, accepted, crit = L.sor_step(X, k=0, omega=omega, cg_tol=1e-6, cg_max=50, solver=api.SOLVER_DIRECT)
        st = L.stats()
    assert accepted == acc
    assert np.linalg.norm(X - Xn) <= 1e-4 * np.linalg.norm(Xn)
    assert f == pytest.approx(fn, rel=1e-4)
    assert 1 <= st["cg_steps"] <= 3  # kappa(A') ~ 10: one or two refinements reach 1e-6
    assert st["cg_maxed"] == 0


@pytest.mark.parametrize("omega", [0.0, 0.5])
def test_converged_run_grid20_matches_oracle(omega):
    rp, ci = synth.grid(20, 20)
    D = _D(rp, ci)
    X0 = synth.initial_layout(400, 2, seed=0)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=omega, tol=1e-4, max_iter=1000)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        L.factor()
        r = L.run(X, trace=True, omega=omega, tol=1e-4, max_iter=1000, solver=api.SOLVER_DIRECT)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))
    assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])


def test_strategies_with_the_direct_solver():
    rp, ci = synth.grid(10, 10)
    D = _D(rp, ci)
    X0 = synth.initial_layout(100, 2, seed=4)
    with api.Layout(rp, ci, dim=2) as L:
        L.factor()
        for strategy in (oracle.OMEGA_PROB, oracle.OMEGA_ENUM):
            ref = oracle.sor_run(D, X0.astype(np.float64), strategy=strategy, seed=42, tol=1e-4, max_iter=60)
            X = X0.copy()
            r = L.run(X, trace=True, strategy=strategy, seed=42, tol=1e-4, max_iter=60, solver=api.SOLVER_DIRECT)
            k = min(5, r.iterations, ref.iterations)
            assert np.array_equal(r.omega[:k], np.array(ref.trace_omega[:k]))
            assert r.stress == pytest.approx(ref.stress, rel=1e-4)


def test_direct_and_cg_runs_agree_and_direct_needs_fewer_solver_steps():
    rp, ci = synth.delaunay(3000, seed=7)
    n = len(rp) - 1
    X0 = synth.initial_layout(n, 2, seed=7)
    with api.Layout(rp, ci, dim=2) as L:
        Xc = X0.copy()
        rc = L.run(Xc, omega=0.5, tol=1e-5, stop=api.STOP_REL_STRESS, max_iter=400)
        sc = L.stats()
        L.factor()
        Xd = X0.copy()
        rd = L.run(Xd, omega=0.5, tol=1e-5, stop=api.STOP_REL_STRESS, max_iter=400, solver=api.SOLVER_DIRECT)
        sd = L.stats()
    assert rd.stress == pytest.approx(rc.stress, rel=1e-4)
    assert sd["cg_maxed"] == 0
    assert sd["cg_steps"] / rd.iterations < sc["cg_steps"] / rc.iterations


def test_adjoint_solve_with_the_direct_solver():
    rp, ci = synth.grid(9, 9)
    ln = _lengths(rp, ci, 1)
    n = len(rp) - 1
    X0 = synth.initial_layout(n, 2, seed=1)
    rng = np.random.default_rng(2)
    Xb = rng.standard_normal((n, 2)).astype(np.float32)
    with api.Layout(rp, ci, dim=2, edge_len=ln) as L:
        X1 = X0.copy()
        L.sor_step(X1, k=0, omega=0.5)
        a, _ = L.sor_step_adjoint(X0, X1, True, 0.5, Xb, cg_tol=1e-7, cg_max=500)
        L.factor()
        b, steps = L.sor_step_adjoint(X0, X1, True, 0.5, Xb, cg_tol=1e-7, cg_max=50, solver=api.SOLVER_DIRECT)
    assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(a)
    assert steps <= 4


def test_direct_solver_needs_a_factor():
    rp, ci = synth.grid(5, 5)
    X = synth.initial_layout(25, 2, seed=0)
    with api.Layout(rp, ci, dim=2) as L:
        with pytest.raises(api.FdError) as e:
            L.run(X.copy(), solver=api.SOLVER_DIRECT)
        assert e.value.status == 1  # FD_ERR_ARG
        L.factor()
        L.run(X.copy(), solver=api.SOLVER_DIRECT, max_iter=3)
        L.factor_release()
        assert L.info()["factored"] == 0
        with pytest.raises(api.FdError):
            L.run(X.copy(), solver=api.SOLVER_DIRECT)
        with pytest.raises(api.FdError):
            L.factor_rows(0, 1)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_graphs(n):
    # one vertex: L^W = 0 and the shift alone is inverted; two and three vertices: K2, P3
    rp, ci = synth.path(n)
    X0 = synth.initial_layout(n, 2, seed=1)
    with api.Layout(rp, ci, dim=2) as L:
        L.factor()
        Ai = L.factor_rows(0, n)
        X = X0.copy()
        r = L.run(X, omega=0.5, tol=1e-6, max_iter=50, solver=api.SOLVER_DIRECT)
    if n == 1:
        assert Ai[0, 0] == pytest.approx(1.0)  # A' = [sigma / n] with sigma = 1 when L^W = 0
        assert r.stress == 0.0
        return
    D = _D(rp, ci)
    assert np.allclose(Ai, oracle.shifted_inverse(D), rtol=1e-5, atol=1e-7)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=0.5, tol=1e-6, max_iter=50)
    assert r.stress == pytest.approx(ref.stress, abs=1e-6 * max(1.0, ref.stress))


def test_weighted_graph_run_matches_oracle():
    rp, ci = synth.grid(10, 10)
    ln = _lengths(rp, ci, 5)
    n = len(rp) - 1
    D = _D(rp, ci, edge_len=ln.astype(np.float64))
    X0 = synth.initial_layout(n, 2, seed=2) * 10.0
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=0.5, tol=1e-5, stop=oracle.STOP_REL_STRESS, max_iter=500)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2, edge_len=ln) as L:
        L.factor()
        r = L.run(X, omega=0.5, tol=1e-5, stop=api.STOP_REL_STRESS, max_iter=500, solver=api.SOLVER_DIRECT)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))
