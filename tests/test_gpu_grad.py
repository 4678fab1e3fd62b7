"""The differentiable form: gradients of the stress through the C ABI,
checked in FP64 against the oracle and central finite differences.

d f / d X is the force kernel (-2 F); d f / d l (edge lengths) sums the pair
derivatives along shortest paths.  Graphs: random geometric graphs in 3-D
with 64 vertices and seeded lengths in [0.5, 2] (the subgraph size of the
differentiable workload's gradient check).
"""
import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


def _weighted_rgg(n, dim, seed):
    for s in range(seed, seed + 50):
        rp, ci, pts = synth.random_geometric(n, dim, 6.0, seed=s)
        if oracle.apsp(rp, ci)[0] == 0:
            break
    rng = np.random.default_rng(s)
    lens = {}
    w = np.empty(len(ci), dtype=np.float32)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, int(ci[e])), max(u, int(ci[e])))
            lens.setdefault(key, np.float32(rng.uniform(0.5, 2.0)))
            w[e] = lens[key]
    return rp, ci, w, pts


@pytest.mark.parametrize("seed", [0, 3])
def test_position_gradient_is_minus_two_forces(seed):
    import torch

    from paper_1711_01228_gb300 import autograd

    rp, ci, w, _ = _weighted_rgg(64, 3, seed)
    D = oracle.apsp(rp, ci, edge_len=w.astype(np.float64))[1]
    X0 = (np.random.default_rng(seed).random((64, 3)) * 3.0).astype(np.float32)
    X = torch.from_numpy(X0).cuda().requires_grad_(True)
    with api.Layout(rp, ci, dim=3, edge_len=w) as L:
        f = autograd.stress(X, L)
        f.backward()
    assert float(f) == pytest.approx(oracle.stress(X0, D), rel=1e-5)
    Xd = X0.astype(np.float64)
    fd = np.zeros_like(Xd)
    h = 1e-6
    for i in range(64):
        for d in range(3):
            Xp, Xm = Xd.copy(), Xd.copy()
            Xp[i, d] += h
            Xm[i, d] -= h
            fd[i, d] = (oracle.stress(Xp, D) - oracle.stress(Xm, D)) / (2 * h)
    g = X.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(fd)


@pytest.mark.parametrize("path", ["shared", "global"])
@pytest.mark.parametrize("seed", [0, 3])
def test_length_gradient_matches_oracle_and_finite_differences(seed, path, monkeypatch):
    # both back-propagation kernels: per-source state in shared memory (n <= 4096)
    # and in global scratch (larger graphs; forced here on the small one)
    if path == "global":
        monkeypatch.setenv("FDLAYOUT_SP_GLOBAL", "1")
    rp, ci, w, _ = _weighted_rgg(64, 3, seed)
    X0 = (np.random.default_rng(seed + 1).random((64, 3)) * 3.0).astype(np.float32)
    with api.Layout(rp, ci, dim=3, edge_len=w) as L:
        f, g = L.length_grad(X0)
    wd = w.astype(np.float64)
    ref = oracle.stress_length_grad(X0, rp, ci, wd)
    assert np.linalg.norm(g - ref) <= 1e-4 * np.linalg.norm(ref)
    # both entries of an edge carry the same value
    n = len(rp) - 1
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(ci[e])
            rev = [k for k in range(rp[v], rp[v + 1]) if ci[k] == u][0]
            assert g[e] == g[rev]
    # central differences of the FP64 stress over re-run shortest paths, on a few edges
    h = 1e-6
    for e in np.random.default_rng(seed).choice(len(ci), 6, replace=False):
        u = int(np.searchsorted(rp, e, side="right") - 1)
        v = int(ci[e])
        idx = [e] + [k for k in range(rp[v], rp[v + 1]) if ci[k] == u]
        wp, wm = wd.copy(), wd.copy()
        wp[idx] += h
        wm[idx] -= h
        fdv = (oracle.stress(X0, oracle.apsp(rp, ci, edge_len=wp)[1]) -
               oracle.stress(X0, oracle.apsp(rp, ci, edge_len=wm)[1])) / (2 * h)
        assert g[e] == pytest.approx(fdv, rel=1e-3, abs=1e-4 * np.abs(ref).max())


def test_autograd_lengths_and_fit():
    import torch

    from paper_1711_01228_gb300 import autograd

    # fit edge lengths (all 1.0 at first) so that the graph distances match a target layout Y
    rp, ci, _, pts = _weighted_rgg(256, 3, 7)
    Y = torch.from_numpy((pts * 10.0).astype(np.float32)).cuda()
    rpt, cit = torch.from_numpy(rp), torch.from_numpy(ci)
    lens = torch.ones(len(ci), dtype=torch.float32, device="cuda", requires_grad=True)
    f0 = autograd.stress_lengths(Y, lens, rpt, cit)
    f0.backward()
    with api.Layout(rp, ci, dim=3, edge_len=np.ones(len(ci), dtype=np.float32)) as L:
        _, g_full = L.length_grad(Y.cpu().numpy())
    # the per-edge sums are added with atomics: equal to FP32 rounding
    assert torch.allclose(lens.grad.cpu(), 0.5 * torch.from_numpy(g_full), rtol=1e-5, atol=0)
    opt = torch.optim.Adam([lens], lr=0.05)
    fs = []
    for _ in range(40):
        opt.zero_grad()
        f = autograd.stress_lengths(Y, lens, rpt, cit)
        f.backward()
        opt.step()
        with torch.no_grad():
            lens.clamp_(min=0.05)
        fs.append(float(f))
    assert fs[-1] < 0.6 * fs[0], fs[::8]
    assert fs[-1] <= 1.05 * min(fs[:10]), fs[::8]


def test_length_gradient_errors():
    rp, ci = synth.grid(5, 5)
    X = synth.initial_layout(25, 2, 0)
    with api.Layout(rp, ci, dim=2) as L:  # no edge lengths
        with pytest.raises(api.FdError) as e:
            L.length_grad(X)
        assert e.value.status == 1
    # a disconnected weighted graph has pairs without a shortest path
    rp, ci = synth.csr_from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)])
    w = np.ones(len(ci), dtype=np.float32)
    with api.Layout(rp, ci, dim=2, edge_len=w, disconnected_policy=1) as L:
        with pytest.raises(api.FdError) as e:
            L.length_grad(synth.initial_layout(6, 2, 0))
        assert e.value.status == 10


@pytest.mark.parametrize("omega,vertex,solver,path", [(0.0, False, 0, "shared"), (0.5, False, 0, "shared"),
                                                      (0.5, True, 0, "shared"), (0.5, False, 1, "shared"),
                                                      (0.5, False, 0, "global")])
def test_unrolled_adjoint_matches_oracle(omega, vertex, solver, path, monkeypatch):
    if path == "global":
        monkeypatch.setenv("FDLAYOUT_SP_GLOBAL", "1")
    """Gradient of a loss on X^K (K = 4 iterations of Algorithm 2, checkpoints
    every 2) in X^0 and in the edge lengths, against the FP64 oracle's adjoint
    (itself pinned by finite differences), with the same acceptance decisions."""
    import torch

    from paper_1711_01228_gb300 import autograd

    rp, ci, w, _ = _weighted_rgg(64, 3, 11)
    n, K = 64, 4
    rng = np.random.default_rng(5)
    X0 = (rng.random((n, 3)) * 3.0).astype(np.float32)
    pairs = np.array([rng.choice(n, 2, replace=False) for _ in range(40)])
    targets = rng.uniform(0.5, 4.0, size=len(pairs))
    Xt = torch.from_numpy(X0).cuda().requires_grad_(True)
    lt = torch.from_numpy(w).cuda().requires_grad_(True)
    m = np.random.default_rng(9).uniform(0.0, 2.0, n).astype(np.float32) if vertex else None
    XK = autograd.unrolled_layout(Xt, lt, torch.from_numpy(rp), torch.from_numpy(ci), K=K, omega=omega, every=2,
                                  cg_tol=1e-7, cg_max=1000, omega_vertex=m, solver=solver)
    pi, pj = torch.from_numpy(pairs[:, 0]).cuda(), torch.from_numpy(pairs[:, 1]).cuda()
    tt = torch.from_numpy(targets).cuda()
    loss = ((XK[pi] - XK[pj]).double().norm(dim=1) - tt).pow(2).sum()
    loss.backward()
    # the GPU's acceptance decisions, from a plain re-run
    accs = []
    with api.Layout(rp, ci, dim=3, edge_len=w) as L:
        if vertex:
            L.set_vertex_omega(m)
        X = X0.copy()
        for k in range(K):
            _, acc, _ = L.sor_step(X, k=k, omega=omega, cg_tol=1e-7, cg_max=1000)
            accs.append(bool(acc))
    D = oracle.apsp(rp, ci, edge_len=w.astype(np.float64))[1]
    m64 = m.astype(np.float64) if vertex else None
    Xs, Zs, acc_ref = oracle.unrolled_run(D, X0.astype(np.float64), K, omega, omega_vertex=m64)
    assert accs == acc_ref
    XKr = Xs[-1]
    gK = np.zeros_like(XKr)
    for (i, j), t in zip(pairs, targets):
        dx = XKr[i] - XKr[j]
        r = np.linalg.norm(dx)
        gK[i] += 2 * (r - t) * dx / r
        gK[j] -= 2 * (r - t) * dx / r
    gX0, Gd = oracle.unrolled_adjoint(D, Xs, Zs, acc_ref, omega, gK, omega_vertex=m64)
    gw = 0.5 * oracle.pair_to_edge_grad(rp, ci, w.astype(np.float64), Gd)
    g_x = Xt.grad.cpu().numpy().astype(np.float64)
    g_l = lt.grad.cpu().numpy().astype(np.float64)
    # Bound: each of the 2K solves (K forward H steps, K adjoint solves) stops
    # at relative residual cg_tol = 1e-7, an error of at most kappa_eff * 1e-7
    # in its solution with kappa_eff (Jacobi-preconditioned L^W on the range)
    # under 100 on these graphs; the iteration map is a contraction, so the
    # errors add: 2K * 100 * 1e-7 = 8e-5 < 1e-4 (FP32 rounding, ~1e-6, below
    # it).  Measured: 1e-6 to 3e-6 with either solver.
    assert np.linalg.norm(g_x - gX0) <= 1e-4 * np.linalg.norm(gX0)
    assert np.linalg.norm(g_l - gw) <= 1e-4 * np.linalg.norm(gw)


def test_length_gradient_above_shared_memory_size():
    """A weighted random geometric graph of 5000 vertices in 3-D (above the
    shared-memory kernel's 4096): the global back-propagation, checked by what
    holds at any size.  (1) Distance rows against scipy's Dijkstra.  (2) d_ij
    is homogeneous of degree 1 in the edge lengths (scaling every length by c
    scales every shortest path by c), so sum_e l_e df/dl_e = sum_{i<j} d_ij
    df/dd_ij with df/dd_ij = -2 r (r - d) / d^3 (Eq. (1), w = d^-2), the right
    side from scipy's distances in FP64.  (3) Central differences of the FP64
    stress (oracle) over scipy's distances for perturbed lengths, two edges."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path

    n = 5000
    rp, ci, pts = synth.random_geometric(n, 3, 6.0, seed=21)
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    ncomp, lab = sp.csgraph.connected_components(A, directed=False)
    keep = np.flatnonzero(lab == np.argmax(np.bincount(lab)))
    sub = A[keep][:, keep].tocsr()
    sub.sort_indices()
    rp, ci = sub.indptr.astype(np.int32), sub.indices.astype(np.int32)
    n = len(rp) - 1
    assert n > 4096
    rng = np.random.default_rng(2)
    lens = {}
    w = np.empty(len(ci), dtype=np.float32)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, int(ci[e])), max(u, int(ci[e])))
            lens.setdefault(key, np.float32(rng.uniform(0.5, 2.0)))
            w[e] = lens[key]
    X = (np.random.default_rng(3).random((n, 3)) * 8.0).astype(np.float32)

    def scipy_D(wv):
        return shortest_path(sp.csr_matrix((wv.astype(np.float64), ci, rp), shape=(n, n)), method="D",
                             directed=False)

    D = scipy_D(w)
    with api.Layout(rp, ci, dim=3, edge_len=w) as L:
        for r in (0, 17, n - 1):
            assert np.allclose(L.distance_rows(r, 1)[0], D[r], rtol=1e-5, atol=0)
        f, g = L.length_grad(X)
    Xd = X.astype(np.float64)
    assert f == pytest.approx(oracle.stress(Xd, D), rel=1e-5)
    iu = np.triu_indices(n, 1)
    r = np.sqrt(((Xd[iu[0]] - Xd[iu[1]]) ** 2).sum(axis=1))
    d = D[iu]
    rhs = float(np.sum(d * (-2.0 * r * (r - d) / d ** 3)))
    lhs = 0.5 * float(np.sum(w.astype(np.float64) * g))  # each edge's two entries carry its derivative
    assert lhs == pytest.approx(rhs, rel=1e-3)
    h = 1e-4
    wd = w.astype(np.float64)
    for e in np.random.default_rng(4).choice(len(ci), 2, replace=False):
        u = int(np.searchsorted(rp, e, side="right") - 1)
        v = int(ci[e])
        idx = [e] + [k for k in range(rp[v], rp[v + 1]) if ci[k] == u]
        wp, wm = wd.copy(), wd.copy()
        wp[idx] += h
        wm[idx] -= h
        fdv = (oracle.stress(Xd, scipy_D(wp)) - oracle.stress(Xd, scipy_D(wm))) / (2 * h)
        assert g[e] == pytest.approx(fdv, rel=2e-3, abs=1e-4 * np.abs(g).max())
