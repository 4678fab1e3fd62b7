"""Pins of the oracle's stress derivatives (no GPU): the gradient in the
positions is -2 F (checked elsewhere); here the derivative with respect to
edge lengths when d_ij is the weighted shortest-path length (Sec. 5.4)."""
import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import synth


def _sym_lengths(rp, ci, rng, lo=0.5, hi=2.0):
    n = len(rp) - 1
    lens = {}
    w = np.empty(len(ci), dtype=np.float64)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, int(ci[e])), max(u, int(ci[e])))
            lens.setdefault(key, rng.uniform(lo, hi))
            w[e] = lens[key]
    return w


def _G(r, d):
    return -2.0 * r * (r - d) / d ** 3


def test_path3_closed_form():
    rp, ci = synth.path(3)  # edges 0-1 (l1) and 1-2 (l2); d_02 = l1 + l2
    l1, l2 = 0.7, 1.9
    w = np.empty(len(ci))
    for u in range(3):
        for e in range(rp[u], rp[u + 1]):
            w[e] = l1 if {u, int(ci[e])} == {0, 1} else l2
    X = np.array([[0.1, 0.2], [1.3, -0.4], [0.5, 2.2]])
    r = lambda i, j: float(np.linalg.norm(X[i] - X[j]))
    want1 = _G(r(0, 1), l1) + _G(r(0, 2), l1 + l2)
    want2 = _G(r(1, 2), l2) + _G(r(0, 2), l1 + l2)
    g = oracle.stress_length_grad(X, rp, ci, w)
    for u in range(3):
        for e in range(rp[u], rp[u + 1]):
            want = want1 if {u, int(ci[e])} == {0, 1} else want2
            assert g[e] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("seed", [0, 2])
def test_length_grad_matches_finite_differences(seed):
    rp, ci, _ = synth.random_geometric(30, 2, 5.0, seed=seed)
    st, _ = oracle.apsp(rp, ci)
    if st != 0:
        pytest.skip("disconnected sample")
    rng = np.random.default_rng(seed)
    w = _sym_lengths(rp, ci, rng)
    X = rng.random((30, 2)) * 3.0
    g = oracle.stress_length_grad(X, rp, ci, w)
    h = 1e-6
    n = len(rp) - 1
    seen = set()
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(ci[e])
            key = (min(u, v), max(u, v))
            if key in seen:
                continue
            seen.add(key)
            idx = [k for k in range(rp[key[0]], rp[key[0] + 1]) if ci[k] == key[1]] + \
                  [k for k in range(rp[key[1]], rp[key[1] + 1]) if ci[k] == key[0]]
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            fp = oracle.stress(X, oracle.apsp(rp, ci, edge_len=wp)[1])
            fm = oracle.stress(X, oracle.apsp(rp, ci, edge_len=wm)[1])
            fd = (fp - fm) / (2 * h)
            assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-7), key


def _loss_and_grad(XK, pairs, targets):
    L = 0.0
    g = np.zeros_like(XK)
    for (i, j), t in zip(pairs, targets):
        dx = XK[i] - XK[j]
        r = float(np.linalg.norm(dx))
        L += (r - t) ** 2
        g[i] += 2.0 * (r - t) * dx / r
        g[j] -= 2.0 * (r - t) * dx / r
    return L, g


@pytest.mark.parametrize("omega,vertex", [(0.0, False), (0.5, False), (0.5, True)])
def test_unrolled_adjoint_matches_finite_differences(omega, vertex):
    # K = 3 iterations of Algorithm 2 on a weighted 16-vertex graph; loss on sampled pair distances;
    # with vertex=True each vertex has its own factor omega_i = omega m_i (Sec. 6)
    rp, ci = synth.grid(4, 4)
    rng = np.random.default_rng(3)
    w = _sym_lengths(rp, ci, rng)
    n, K = 16, 3
    X0 = rng.random((n, 2)) * 2.0
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(12)]
    targets = rng.uniform(0.5, 3.0, size=len(pairs))
    m = np.random.default_rng(9).uniform(0.0, 2.0, n) if vertex else None

    def run(X0_, w_):
        D = oracle.apsp(rp, ci, edge_len=w_)[1]
        Xs, Zs, acc = oracle.unrolled_run(D, X0_, K, omega, omega_vertex=m)
        return Xs, Zs, acc, D

    Xs, Zs, acc, D = run(X0, w)
    L0, gK = _loss_and_grad(Xs[-1], pairs, targets)
    gX0, Gd = oracle.unrolled_adjoint(D, Xs, Zs, acc, omega, gK, omega_vertex=m)
    gw = oracle.pair_to_edge_grad(rp, ci, w, Gd)
    h = 1e-6
    checked = 0
    for i in range(n):
        for d in range(2):
            Xp, Xm = X0.copy(), X0.copy()
            Xp[i, d] += h
            Xm[i, d] -= h
            rp_, rm_ = run(Xp, w), run(Xm, w)
            if rp_[2] != acc or rm_[2] != acc:
                continue  # an acceptance decision flipped: not differentiable here
            fd = (_loss_and_grad(rp_[0][-1], pairs, targets)[0] - _loss_and_grad(rm_[0][-1], pairs, targets)[0]) / (2 * h)
            assert gX0[i, d] == pytest.approx(fd, rel=1e-4, abs=1e-6 * max(1.0, abs(L0)))
            checked += 1
    assert checked >= 24
    seen = set()
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(ci[e])
            key = (min(u, v), max(u, v))
            if key in seen:
                continue
            seen.add(key)
            idx = [k for k in range(rp[key[0]], rp[key[0] + 1]) if ci[k] == key[1]] + \
                  [k for k in range(rp[key[1]], rp[key[1] + 1]) if ci[k] == key[0]]
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            rp_, rm_ = run(X0, wp), run(X0, wm)
            if rp_[2] != acc or rm_[2] != acc:
                continue
            fd = (_loss_and_grad(rp_[0][-1], pairs, targets)[0] - _loss_and_grad(rm_[0][-1], pairs, targets)[0]) / (2 * h)
            assert gw[e] == pytest.approx(fd, rel=1e-4, abs=1e-6 * max(1.0, abs(L0))), key
