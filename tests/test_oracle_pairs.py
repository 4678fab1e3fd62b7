"""Pins of the oracle's pair functions: stress (Eq. (1)), L^X X, L^W P and
the force (L^X - L^W) X (Prop. 2.1).

Pins: closed forms on 2-4 vertex graphs, the trace form g(X, X) of Prop. 2.1,
the majorization inequality, central finite differences of scalar sums, and
invariances under translation, rotation and reflection.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import synth


def _dense_D(rp, ci):
    st, D = oracle.apsp(rp, ci, policy=1)
    return D


def _rand_graph(n=24, seed=0):
    rp, ci = synth.erdos_renyi(n, 4.0, seed=seed)
    return _dense_D(rp, ci)


def test_stress_two_vertices():
    D = _dense_D(*synth.path(2))
    for r in (0.3, 1.0, 2.5):
        X = np.array([[0.0, 0.0], [r, 0.0]])
        assert oracle.stress(X, D) == pytest.approx((r - 1.0) ** 2, abs=1e-15)


def test_stress_path_and_triangle_zero():
    D = _dense_D(*synth.path(3))
    assert oracle.stress(np.array([[0.0], [1.0], [2.0]]), D) == pytest.approx(0.0, abs=1e-15)
    D = _dense_D(*synth.complete(3))
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    assert oracle.stress(X, D) == pytest.approx(0.0, abs=1e-15)


def test_stress_square_and_star():
    # C4 laid out as a square of side s: 4 pairs at d=1, 2 diagonals at d=2.
    D = _dense_D(*synth.cycle(4))
    s = 1.3
    X = np.array([[0, 0], [s, 0], [s, s], [0, s]], dtype=np.float64)
    expect = 4 * (s - 1) ** 2 + 2 * (math.sqrt(2) * s - 2) ** 2 / 4
    assert oracle.stress(X, D) == pytest.approx(expect, rel=1e-14)
    # K_{1,3}: centre + 3 leaves at 120 degrees, radius r.
    D = _dense_D(*synth.star(3))
    r = 0.8
    ang = np.array([0, 2 * math.pi / 3, 4 * math.pi / 3])
    X = np.vstack([[0, 0], np.stack([r * np.cos(ang), r * np.sin(ang)], 1)])
    expect = 3 * (r - 1) ** 2 + 3 * (math.sqrt(3) * r - 2) ** 2 / 4
    assert oracle.stress(X, D) == pytest.approx(expect, rel=1e-14)


def test_trace_form_equals_stress():
    # Prop. 2.1: f(X) = g(X, X).
    D = _rand_graph()
    rng = np.random.default_rng(1)
    for dim in (1, 2, 3):
        X = rng.random((D.shape[0], dim))
        assert oracle.majorant(X, X, D) == pytest.approx(oracle.stress(X, D), rel=1e-12)


def test_majorant_dominates():
    # Prop. 2.1: f(X) <= g(X, Y) for all X, Y.
    D = _rand_graph(seed=2)
    rng = np.random.default_rng(2)
    for _ in range(10):
        X = rng.random((D.shape[0], 2))
        Y = rng.random((D.shape[0], 2))
        assert oracle.stress(X, D) <= oracle.majorant(X, Y, D) + 1e-12


def _fd_grad(fun, X, h=1e-6):
    G = np.zeros_like(X)
    for idx in np.ndindex(*X.shape):
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        G[idx] = (fun(Xp) - fun(Xm)) / (2 * h)
    return G


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_forces_are_minus_half_gradient(dim):
    D = _rand_graph(n=16, seed=dim)
    X = np.random.default_rng(dim).random((16, dim))
    G = _fd_grad(lambda Y: oracle.stress(Y, D), X)
    F = oracle.forces(X, D)
    assert np.allclose(-2.0 * F, G, rtol=1e-6, atol=1e-7 * np.abs(G).max())


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_lw_matvec_is_gradient_of_dirichlet_sum(dim):
    # sum_{i<j} w_ij ||p_i - p_j||^2 = tr(P^T L^W P); its gradient is 2 L^W P.
    D = _rand_graph(n=14, seed=10 + dim)
    P = np.random.default_rng(dim).random((14, dim))
    iu = np.triu_indices(14, 1)

    def dirichlet(Y):
        diff = Y[iu[0]] - Y[iu[1]]
        return float(np.sum(np.sum(diff * diff, axis=1) / D[iu] ** 2))

    G = _fd_grad(dirichlet, P)
    assert np.allclose(2.0 * oracle.lw_matvec(P, D), G, rtol=1e-6, atol=1e-7 * np.abs(G).max())
    assert np.allclose(oracle.lw_matvec(np.ones((14, dim)), D), 0.0, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_rhs_is_gradient_of_weighted_distance_sum(dim):
    # sum_{i<j} w_ij d_ij ||x_i - x_j||; its gradient is L^X X.
    D = _rand_graph(n=14, seed=20 + dim)
    X = np.random.default_rng(dim).random((14, dim))
    iu = np.triu_indices(14, 1)

    def wdr(Y):
        r = np.sqrt(np.sum((Y[iu[0]] - Y[iu[1]]) ** 2, axis=1))
        return float(np.sum(r / D[iu]))

    G = _fd_grad(wdr, X)
    assert np.allclose(oracle.rhs(X, D), G, rtol=1e-6, atol=1e-7 * np.abs(G).max())


def test_sums_vanish_and_rows_agree():
    D = _rand_graph(n=30, seed=4)
    X = np.random.default_rng(4).random((30, 2))
    b, F = oracle.rhs(X, D), oracle.forces(X, D)
    assert np.allclose(b.sum(0), 0.0, atol=1e-12)
    assert np.allclose(F.sum(0), 0.0, atol=1e-12)
    for i in (0, 13, 29):
        assert np.allclose(oracle.force_row(X, i, D[i]), F[i], rtol=1e-14, atol=1e-14)
        assert np.allclose(oracle.rhs_row(X, i, D[i]), b[i], rtol=1e-14, atol=1e-14)


def test_invariances():
    D = _rand_graph(n=20, seed=5)
    X = np.random.default_rng(5).random((20, 2))
    f, F, b = oracle.stress(X, D), oracle.forces(X, D), oracle.rhs(X, D)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    refl = np.array([[1.0, 0.0], [0.0, -1.0]])
    for Q in (R, refl):
        Y = X @ Q.T + np.array([3.0, -2.0])
        assert oracle.stress(Y, D) == pytest.approx(f, rel=1e-12)
        assert np.allclose(oracle.forces(Y, D), F @ Q.T, rtol=1e-10, atol=1e-12)
        assert np.allclose(oracle.rhs(Y, D), b @ Q.T, rtol=1e-10, atol=1e-12)


def test_coincident_vertices():
    # l^Y_ij = 0 when y_i = y_j (Prop. 2.1); the stress term is then w d^2.
    D = _dense_D(*synth.path(3))
    X = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    b = oracle.rhs(X, D)
    assert np.all(np.isfinite(b))
    # vertex 0 only feels vertex 2 (d = 2): w d (x0 - x2)/r = (1/2)(-1, 0)
    assert np.allclose(b[0], [-0.5, 0.0])
    assert oracle.stress(X, D) == pytest.approx(1.0 + 0.0 + (1.0 - 2.0) ** 2 / 4.0)


def test_force_magnitude_bounds_and_equalities():
    # A_ic = sum_j |w_ij (d_ij/r_ij - 1)(x_ic - x_jc)|, the scale of the
    # per-element force tolerances.  Pins: with one term (K2) A = |F|; |F| <= A
    # always (triangle inequality), strictly for a row whose terms mix signs;
    # A = |F| for a row whose terms share one sign.
    D2 = _dense_D(*synth.path(2))
    X2 = np.array([[0.1, 0.3], [1.7, -0.2]])
    assert np.allclose(oracle.force_abs(X2, D2), np.abs(oracle.forces(X2, D2)), rtol=1e-15, atol=0)
    D = _dense_D(*synth.delaunay(40, seed=6))
    X = np.random.default_rng(6).random((40, 2)) * 3.0
    A, F = oracle.force_abs(X, D), oracle.forces(X, D)
    assert np.all(np.abs(F) <= A * (1 + 1e-12))
    assert np.any(np.abs(F) < 0.5 * A)
    # vertex 0 at the origin, the others on the positive x axis beyond their
    # ideal distances: every term of row 0 is w (d/r - 1)(0 - x_j) > 0
    n = 6
    Dp = _dense_D(*synth.path(n))
    Xl = np.zeros((n, 2))
    Xl[1:, 0] = 2.0 * np.arange(1, n) + 0.5
    A0 = oracle.force_row_abs(Xl, 0, Dp[0])
    F0 = oracle.force_row(Xl, 0, Dp[0])
    assert F0[0] > 0 and A0[0] == pytest.approx(F0[0], rel=1e-15) and A0[1] == 0.0
