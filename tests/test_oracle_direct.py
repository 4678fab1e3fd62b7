"""Pins of the oracle's shifted inverse, the matrix the direct solver of
Eq. (2-5) applies: A'^-1 with A' = L^W + (sigma/n) 1 1^T, sigma = mean_i s_i.

Pins: closed forms on K2 and on the complete graph K5 (eigenvalues sigma on
1 and n on its complement); A'^-1 1 = 1 / sigma; for a zero-sum right-hand
side, A'^-1 b and the pinned Cholesky solve of Eq. (2-5) (a different
method) differ by a translation; the conditioning that makes FP32 usable.
"""
import numpy as np

import oracle
from paper_1711_01228_gb300 import synth


def _D(rp, ci):
    st, D = oracle.apsp(rp, ci, policy=1)
    return D


def test_K2_closed_form():
    # L^W = [[1, -1], [-1, 1]], sigma = 1: A' = [[1.5, -0.5], [-0.5, 1.5]]
    Ai = oracle.shifted_inverse(_D(*synth.path(2)))
    assert np.allclose(Ai, [[0.75, 0.25], [0.25, 0.75]], rtol=0, atol=1e-15)


def test_complete_graph_closed_form():
    # K5, d = 1: L^W = 5 I - J, sigma = 4, A' = 5 I - J + (4/5) J = 5 I - J / 5.
    # On 1: eigenvalue 4; on its complement: 5.  A'^-1 = I/5 + (1/4 - 1/5) J/5.
    Ai = oracle.shifted_inverse(_D(*synth.complete(5)))
    ref = np.eye(5) / 5 + (0.25 - 0.2) * np.ones((5, 5)) / 5
    assert np.allclose(Ai, ref, rtol=0, atol=1e-15)


def test_constant_vector_and_symmetry():
    D = _D(*synth.delaunay(80, seed=1))
    Ai = oracle.shifted_inverse(D)
    sigma = np.trace(oracle.lw_dense(D)) / 80
    assert np.allclose(Ai @ np.ones(80), np.ones(80) / sigma, rtol=1e-12, atol=0)
    assert np.allclose(Ai, Ai.T, rtol=0, atol=1e-14)


def test_zero_sum_solve_is_the_pinned_solve_up_to_translation():
    for rp, ci in (synth.grid(7, 9), synth.erdos_renyi(90, 4.0, seed=2), synth.random_binary_tree(63, seed=3)):
        n = len(rp) - 1
        D = _D(rp, ci)
        X = np.random.default_rng(n).random((n, 2))
        b = oracle.rhs(X, D)
        Zs = oracle.shifted_inverse(D) @ b
        Zp = oracle.PinnedSolver(D).solve(b)
        t = Zs - Zp
        assert np.abs(t - t[0]).max() <= 1e-10 * np.abs(Zp).max()
        assert np.abs(Zs.sum(axis=0)).max() <= 1e-10 * np.abs(Zs).max()


def test_shift_keeps_the_conditioning_of_L():
    # the pinned matrix is ~n times worse conditioned; the shifted one keeps
    # lambda_max / lambda_2 of L^W (Prop. 2.1: L^W is positive semi-definite
    # with the single null vector 1 on a connected graph)
    D = _D(*synth.grid(12, 12))
    L = oracle.lw_dense(D)
    lam = np.linalg.eigvalsh(L)
    ev = 1.0 / np.linalg.eigvalsh(oracle.shifted_inverse(D))
    kappa_shift = ev.max() / ev.min()
    assert kappa_shift <= lam[-1] / lam[1] * (1 + 1e-9)
    pinned = np.linalg.eigvalsh(L[1:, 1:])
    assert pinned[-1] / pinned[0] > 20 * kappa_shift
