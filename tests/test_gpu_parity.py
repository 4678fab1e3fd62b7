"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances, from the arithmetic of the kernels:
  distances       bit-exact (integer hop counts); 1e-5 relative for float lengths
                  (FP32 sums along a path against FP64 Dijkstra)
  stress          1e-5 relative (FP32 pair terms, FP32 sums of <= 128 terms, FP64 above)
  forces          1e-5 relative, Frobenius norm over all vertices (per-element
                  error about 32 eps32 sum |terms|, ~1e-6 at random layouts)
  one SOR step    1e-4 relative on the layout (CG stops at relative residual 1e-6;
                  the layout error is at most kappa_eff times that, kappa_eff <= 100)
  converged run   1e-4 relative on final stress, iterations within 2 % (at least 1)
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


def _dense(rp, ci, policy=1, edge_len=None):
    st, D = oracle.apsp(rp, ci, edge_len=edge_len, policy=policy)
    return D


GRAPHS = {
    "path2": lambda: synth.path(2),
    "k3": lambda: synth.complete(3),
    "grid20": lambda: synth.grid(20, 20),
    "er300": lambda: synth.erdos_renyi(300, 4.0, seed=1),
    "tree383": lambda: synth.random_binary_tree(383, seed=2),
    "delaunay1000": lambda: synth.delaunay(1000, seed=3),
    "ba1500": lambda: synth.barabasi_albert(1500, 3, seed=4),
    "rgg2049": lambda: synth.random_geometric(2049, 2, 6.0, seed=5)[:2],
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_distances_bit_exact(name):
    rp, ci = GRAPHS[name]()
    D = _dense(rp, ci)
    n = len(rp) - 1
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        got = L.distance_rows(0, n)
        info = L.info()
    assert np.array_equal(got, D)
    assert info["diameter"] == int(D.max()) or info["disconnected"] == 1


def _short_and_long_path():
    # vertex 0 on a 3-vertex path (eccentricity 2), beside a 300-vertex path
    # (diameter 299 would need float codes; 200 vertices: 199 fits a byte):
    # searches from the long path run far deeper than vertex 0's component
    edges = [(0, 1), (1, 2)] + [(i, i + 1) for i in range(3, 202)]
    return synth.csr_from_edges(203, edges)


def _er_with_hubs():
    # an Erdos-Renyi graph (n = 2000, mean degree 4) with two hubs joined to
    # 700 and 300 random vertices: degrees above 256, split over several warps
    rp, ci = synth.erdos_renyi(2000, 4.0, seed=3)
    rng = np.random.default_rng(5)
    edges = {(min(u, int(v)), max(u, int(v))) for u in range(2000) for v in ci[rp[u]:rp[u + 1]] if u != v}
    for hub, k in ((17, 700), (1500, 300)):
        for v in rng.choice(2000, k, replace=False):
            if int(v) != hub:
                edges.add((min(hub, int(v)), max(hub, int(v))))
    return synth.csr_from_edges(2000, sorted(edges))


WIDE_GRAPHS = dict(GRAPHS, star700=lambda: synth.star(700), path300=lambda: synth.path(300),
                   paths203=_short_and_long_path, erhubs2000=_er_with_hubs)


@pytest.mark.parametrize("name", ["path2", "k3", "grid20", "er300", "tree383", "ba1500", "rgg2049", "star700",
                                  "path300", "paths203", "erhubs2000"])
def test_distances_bit_exact_level_synchronous(name, monkeypatch):
    # the 256-source search over all CTAs (a grid barrier per level), forced at
    # sizes the dense oracle holds: one ragged batch (n < 256), several batches
    # with a ragged last one, a disconnected graph, a deep tree (many levels),
    # vertices of degree above 16 (pulled by a warp each: the hubs of ba1500;
    # above 256, split over several warps: the centre of star700, the two
    # hubs of erhubs2000), float codes (path300: diameter 299 > 254), and
    # levels past the frontiers kept for the end-of-batch codes (paths203:
    # those codes are written as reached and merged with the decoded ones)
    rp, ci = WIDE_GRAPHS[name]()
    D = _dense(rp, ci)
    n = len(rp) - 1
    monkeypatch.setenv("FDLAYOUT_BFS_WIDE", "1")
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        got = L.distance_rows(0, n)
        info = L.info()
    assert info["bfs_sources"] == 256
    assert np.array_equal(got, D)
    assert info["diameter"] == int(D.max()) or info["disconnected"] == 1
    monkeypatch.setenv("FDLAYOUT_BFS_WIDE", "0")
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        assert L.info()["bfs_sources"] == 64
        assert np.array_equal(L.distance_rows(0, n), got)


def test_distances_weighted():
    rp, ci = synth.delaunay(300, seed=7)
    rng = np.random.default_rng(0)
    n = len(rp) - 1
    lens = {}
    w = np.empty(len(ci), dtype=np.float32)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, ci[e]), max(u, ci[e]))
            lens.setdefault(key, np.float32(rng.uniform(0.5, 2.0)))
            w[e] = lens[key]
    D = _dense(rp, ci, edge_len=w.astype(np.float64))
    with api.Layout(rp, ci, dim=2, edge_len=w) as L:
        got = L.distance_rows(0, n)
        assert L.info()["code_bytes"] == 4
    assert np.allclose(got, D, rtol=1e-5, atol=0)


def test_disconnected_policy():
    rp, ci = synth.erdos_renyi(200, 1.5, seed=3)
    with pytest.raises(api.FdError) as e:
        api.Layout(rp, ci, dim=2, disconnected_policy=0)
    assert e.value.status == 3
    D = _dense(rp, ci, policy=1)
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        assert L.info()["disconnected"] == 1
        assert np.array_equal(L.distance_rows(0, len(rp) - 1), D)


CASES = [("path2", 1), ("path2", 2), ("k3", 3), ("grid20", 2), ("er300", 2), ("er300", 3), ("tree383", 1),
         ("delaunay1000", 2), ("ba1500", 3), ("rgg2049", 2)]


@pytest.mark.parametrize("name,dim", CASES)
def test_energy_and_forces(name, dim):
    rp, ci = GRAPHS[name]()
    n = len(rp) - 1
    D = _dense(rp, ci)
    X = synth.initial_layout(n, dim, seed=11) * 3.0
    f_ref = oracle.stress(X, D)
    F_ref = oracle.forces(X, D)
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        f = L.energy(X)
        F = L.forces(X)
    assert f == pytest.approx(f_ref, rel=1e-5)
    err = np.linalg.norm(F.astype(np.float64) - F_ref)
    assert err <= 1e-5 * np.linalg.norm(F_ref) + 1e-12


def test_torch_device_pointers():
    import torch

    rp, ci = synth.delaunay(700, seed=2)
    n = len(rp) - 1
    D = _dense(rp, ci)
    X = synth.initial_layout(n, 2, seed=1)
    Xt = torch.from_numpy(X).cuda()
    with api.Layout(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), dim=2) as L:
        f = L.energy(Xt)
        F = L.forces(Xt)
        assert F.is_cuda
    assert f == pytest.approx(oracle.stress(X, D), rel=1e-5)
    F_ref = oracle.forces(X, D)
    assert np.linalg.norm(F.cpu().numpy() - F_ref) <= 1e-5 * np.linalg.norm(F_ref)


def test_coincident_and_nonfinite():
    rp, ci = synth.path(3)
    D = _dense(rp, ci)
    X = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]], dtype=np.float32)
    with api.Layout(rp, ci, dim=2) as L:
        assert L.energy(X) == pytest.approx(oracle.stress(X, D), rel=1e-6)
        F = L.forces(X)
        assert np.allclose(F, oracle.forces(X, D), atol=1e-6)
        Xb = X.copy()
        Xb[1, 0] = np.nan
        with pytest.raises(api.FdError) as e:
            L.energy(Xb)
        assert e.value.status == 4


@pytest.mark.parametrize("name,dim,omega", [("grid20", 2, 0.5), ("delaunay1000", 2, 1.0), ("er300", 3, 0.5),
                                            ("tree383", 1, 0.0)])
def test_one_sor_step(name, dim, omega):
    rp, ci = GRAPHS[name]()
    n = len(rp) - 1
    D = _dense(rp, ci)
    X0 = synth.initial_layout(n, dim, seed=5)
    Xn, fn, acc, om, fZ = oracle.sor_step(X0.astype(np.float64), D, omega)
    X = X0.copy()
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        f, accepted, crit = L.sor_step(X, k=0, omega=omega, cg_tol=1e-6, cg_max=500)
    assert accepted == acc
    assert np.linalg.norm(X - Xn) <= 1e-4 * np.linalg.norm(Xn)
    assert f == pytest.approx(fn, rel=1e-4)
    crit_ref = oracle.criterion(oracle.STOP_REL_DISP, X0.astype(np.float64), Xn, 0, 0)
    assert crit == pytest.approx(crit_ref, rel=1e-3)


@pytest.mark.parametrize("omega", [0.0, 0.5])
def test_converged_run_grid20(omega):
    # 20x20 grid, X^0 uniform in [0,1]^2 from seed 0, relative displacement 1e-4, max 1000 iterations
    rp, ci = synth.grid(20, 20)
    D = _dense(rp, ci)
    X0 = synth.initial_layout(400, 2, seed=0)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=omega, tol=1e-4, max_iter=1000)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        r = L.run(X, trace=True, omega=omega, tol=1e-4, max_iter=1000)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))
    assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])  # Prop. 2.2 / line 6
    assert r.trace_f[0] == pytest.approx(ref.trace_f[0], rel=1e-5)


def test_extended_trace_matches_oracle():
    # f(H(X^k)) and f of the extrapolated candidate per iteration (lines 4-6 of
    # Algorithm 2), against the oracle's trace_fH; the times increase
    rp, ci = synth.grid(12, 12)
    D = _dense(rp, ci)
    X0 = synth.initial_layout(144, 2, seed=6)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=1.0, tol=1e-5, max_iter=60)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        r = L.run(X, trace=True, omega=1.0, tol=1e-5, max_iter=60)
    k = min(10, r.iterations, ref.iterations)
    assert np.allclose(r.f_h[:k], np.array(ref.trace_fH[:k]), rtol=1e-4, atol=0)
    for i in range(r.iterations):
        # line 6: the kept stress is the extrapolated one if accepted, else f(H(X^k))
        kept = r.f_extrapolated[i] if r.accepted[i] else r.f_h[i]
        assert r.trace_f[i + 1] == kept
        assert r.accepted[i] == (r.f_extrapolated[i] <= r.f_h[i])
    assert np.all(np.diff(r.t_ms) > 0) and r.t_ms[0] > 0
    assert r.t_ms[-1] <= r.stats["kernel_ms"] * 1.01 + 0.05


def test_probabilistic_strategy_matches_oracle_sequence():
    rp, ci = synth.grid(10, 10)
    D = _dense(rp, ci)
    X0 = synth.initial_layout(100, 2, seed=3)
    ref = oracle.sor_run(D, X0.astype(np.float64), strategy=oracle.OMEGA_PROB, seed=42, tol=1e-4, max_iter=30)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        r = L.run(X, trace=True, strategy=api.OMEGA_PROB, seed=42, tol=1e-4, max_iter=30)
    k = min(r.iterations, ref.iterations)
    assert np.array_equal(r.omega[:k], np.array(ref.trace_omega[:k]))


@pytest.mark.parametrize("ctas", [1, 3, 7])
def test_many_tasks_per_cta(ctas, monkeypatch):
    # With few CTAs every CTA walks many tasks and tiles: the prefetch chain,
    # the task hand-over and the partial sums must not depend on the grid.
    monkeypatch.setenv("FDLAYOUT_MAX_CTAS", str(ctas))
    rp, ci = GRAPHS["delaunay1000"]()
    n = len(rp) - 1
    D = _dense(rp, ci)
    X0 = synth.initial_layout(n, 2, seed=8)
    with api.Layout(rp, ci, dim=2) as L:
        assert L.info()["grid"] == ctas
        assert L.energy(X0) == pytest.approx(oracle.stress(X0, D), rel=1e-5)
        F = L.forces(X0)
        F_ref = oracle.forces(X0, D)
        assert np.linalg.norm(F - F_ref) <= 1e-5 * np.linalg.norm(F_ref)
        X = X0.copy()
        f, acc, crit = L.sor_step(X, k=0, omega=0.5)
    Xn, fn, accn, _, _ = oracle.sor_step(X0.astype(np.float64), D, 0.5)
    assert acc == accn
    assert np.linalg.norm(X - Xn) <= 1e-4 * np.linalg.norm(Xn)


def test_enumerating_strategy_matches_oracle():
    # Sec. 5.2.2: omega = argmin of f over {0, 0.5, ..., 9}, ties to the smaller omega
    rp, ci = synth.grid(10, 10)
    D = _dense(rp, ci)
    X0 = synth.initial_layout(100, 2, seed=4)
    ref = oracle.sor_run(D, X0.astype(np.float64), strategy=oracle.OMEGA_ENUM, tol=1e-4, max_iter=60)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        r = L.run(X, trace=True, strategy=api.OMEGA_ENUM, tol=1e-4, max_iter=60)
    k = min(5, r.iterations, ref.iterations)
    assert np.array_equal(r.omega[:k], np.array(ref.trace_omega[:k]))
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))
    assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])


def test_barrier_timeout_reports_status_and_context_survives(monkeypatch):
    # Failure detection without a GPU fault: the grid-barrier waits get a 1 ns
    # limit, run out, and the kernel returns FD_ERR_TIMEOUT (the copy waits keep
    # their own limit, so no CTA leaves with a copy in flight).  The next handle
    # on the same device still computes correctly.
    rp, ci = synth.grid(30, 30)
    n = len(rp) - 1
    X = synth.initial_layout(n, 2, seed=2)
    monkeypatch.setenv("FDLAYOUT_BARRIER_TIMEOUT_NS", "1")
    with api.Layout(rp, ci, dim=2) as L:
        with pytest.raises(api.FdError) as e:
            L.energy(X)
        assert e.value.status == 7
        with pytest.raises(api.FdError) as e:
            L.run(X.copy(), omega=0.5, tol=1e-4, max_iter=5)
        assert e.value.status == 7
        assert api.lib().fd_last_error(L._h) == 7
    monkeypatch.delenv("FDLAYOUT_BARRIER_TIMEOUT_NS")
    D = _dense(rp, ci)
    with api.Layout(rp, ci, dim=2) as L:
        assert L.energy(X) == pytest.approx(oracle.stress(X, D), rel=1e-5)
        Xr = X.copy()
        r = L.run(Xr, omega=0.5, tol=1e-4, max_iter=20)
        assert r.iterations > 0


@pytest.mark.parametrize("seed", [0, 3])
def test_fig4_graph_runs_match_oracle(seed):
    # the paper's Fig. 4 (left) graph, Algorithm 2 at omega = 0.5 to relative stress decrease 1e-6
    import test_oracle_fig4

    rp, ci, _ = test_oracle_fig4.load_fig4()
    D = _dense(rp, ci)
    X0 = synth.initial_layout(179, 2, seed)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=0.5, tol=1e-6, stop=oracle.STOP_REL_STRESS, max_iter=5000)
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        r = L.run(X, omega=0.5, tol=1e-6, stop=api.STOP_REL_STRESS, max_iter=5000)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))


@pytest.mark.parametrize("dim", [2, 3])
def test_invariance_under_rigid_motion(dim):
    # f depends only on distances (Eq. (1)): translation and rotation leave it unchanged and rotate F
    rp, ci = GRAPHS["delaunay1000"]()
    n = len(rp) - 1
    rng = np.random.default_rng(3)
    X = synth.initial_layout(n, dim, seed=4).astype(np.float64) * 3.0
    Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
    t = rng.normal(size=dim) * 5.0
    Y = X @ Q.T + t
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        fX, fY = L.energy(X.astype(np.float32)), L.energy(Y.astype(np.float32))
        FX = L.forces(X.astype(np.float32)).astype(np.float64)
        FY = L.forces(Y.astype(np.float32)).astype(np.float64)
    assert fY == pytest.approx(fX, rel=1e-5)
    assert np.linalg.norm(FY - FX @ Q.T) <= 1e-4 * np.linalg.norm(FX)


@pytest.mark.parametrize("tps", ["1", "2"])
def test_stage_shapes_agree_with_oracle(tps, monkeypatch):
    # one or two consecutive tiles per pipeline stage (the two-tile kernel serves
    # uint8 codes with a small table): a graph of 6 blocks with a ragged last
    # block, so that tasks end on odd and even tile counts, steps wrap past the
    # last block, and few CTAs walk many steps.  A Delaunay mesh, whose run
    # converges (111 iterations in FP64), so that the converged-run bounds
    # apply; a capped run (the 700-vertex BA graph stops at 1000 iterations
    # with its stress still falling 5e-6 per iteration) compares trajectories,
    # not layouts.
    monkeypatch.setenv("FDLAYOUT_TPS", tps)
    monkeypatch.setenv("FDLAYOUT_MAX_CTAS", "5")
    rp, ci = synth.delaunay(700, seed=9)
    n = len(rp) - 1
    D = _dense(rp, ci)
    X0 = synth.initial_layout(n, 2, seed=2)
    with api.Layout(rp, ci, dim=2) as L:
        assert L.info()["tiles_per_stage"] == int(tps)
        assert L.energy(X0) == pytest.approx(oracle.stress(X0, D), rel=1e-5)
        F = L.forces(X0).astype(np.float64)
        A = oracle.force_abs(X0, D)
        assert np.all(np.abs(F - oracle.forces(X0, D)) <= 1e-5 * A + 1e-30)
        X = X0.copy()
        r = L.run(X, trace=True, omega=0.5, tol=1e-4, max_iter=1000)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=0.5, tol=1e-4, max_iter=1000)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("solver", [api.SOLVER_CG, api.SOLVER_DIRECT])
def test_h_step_start_from_previous_step(dim, solver):
    """Inside one launch, L^W X^{k+1} at the start of an H step comes from the
    previous H step's right-hand side and residuals (L^W z = B - R, L^W X^k =
    B - R0) instead of an all-pairs pass, except at every 16th iteration.  One
    launch of 20 iterations against 20 launches of one iteration each (every one
    of which runs the pass): the same acceptance decisions, layouts within 1e-4
    relative, final stresses within 1e-5 of each other, and both within the
    converged-run bound 1e-4 of the FP64 oracle's run (20 iterations of H steps
    solved to CG's 1e-6 drift from the exact solves by a few 1e-5)."""
    rp, ci = synth.delaunay(1200, seed=31)
    n = len(rp) - 1
    st, D = oracle.apsp(rp, ci)
    X0 = synth.initial_layout(n, dim, seed=4)
    K = 20
    with api.Layout(rp, ci, dim=dim) as L:
        if solver == api.SOLVER_DIRECT:
            L.factor()
        Xa = X0.copy()
        ra = L.run(Xa, trace=True, omega=0.5, tol=0.0, max_iter=K, solver=solver)
        assert ra.iterations == K
        Xb = X0.copy()
        acc_b = []
        for k in range(K):
            f, acc, _ = L.sor_step(Xb, k=k, omega=0.5, solver=solver)
            acc_b.append(bool(acc))
    assert list(map(bool, ra.accepted[:K])) == acc_b
    assert np.linalg.norm(Xa - Xb) <= 1e-4 * np.linalg.norm(Xb)
    assert ra.stress == pytest.approx(f, rel=1e-5)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=0.5, tol=0.0, max_iter=K)
    assert ra.stress == pytest.approx(ref.stress, rel=1e-4)
    assert f == pytest.approx(ref.stress, rel=1e-4)
