"""Pins of the oracle's per-vertex relaxation factors (Sec. 6, first item of
further work: vertex i is relaxed by its own stride omega_i,
x~_i = x_i^{k+1} + omega_i (x_i^{k+1} - x_i^k)); the library takes
omega_i = omega m_i.

Pins: the candidate worked out by hand on K2 (catches a factor applied to
the wrong vertex or with the wrong sign); constant factors reduce to Eq. (10)
with a single omega; m = 0 is Algorithm 1; relabelling the vertices
(vertex 0, the pinned one, kept) relabels the run; the acceptance chain of
line 6 and Prop. 2.2 still holds.
"""
import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import synth


def _D(rp, ci):
    st, D = oracle.apsp(rp, ci, policy=1)
    return D


def test_K2_candidate_by_hand():
    # K2 with d = 1, x_0 = (1, 0), x_1 = (4, 0).  H pins vertex 0 at the
    # origin and puts vertex 1 at unit distance along x_1 - x_0: z = (0,0), (1,0).
    D = _D(*synth.path(2))
    X = np.array([[1.0, 0.0], [4.0, 0.0]])
    Z = oracle.H(X, D)
    assert np.allclose(Z, [[0.0, 0.0], [1.0, 0.0]], atol=1e-15)
    # omega = 0.5, m = (0.6, 0.2): omega_0 = 0.3, omega_1 = 0.1
    #   x~_0 = (0,0) + 0.3 ((0,0) - (1,0)) = (-0.3, 0)
    #   x~_1 = (1,0) + 0.1 ((1,0) - (4,0)) = ( 0.7, 0)
    Xt = oracle.extrapolate(Z, X, 0.5, np.array([0.6, 0.2]))
    assert np.allclose(Xt, [[-0.3, 0.0], [0.7, 0.0]], atol=1e-15)
    # without factors, Eq. (10): (1.5) z - 0.5 x
    assert np.allclose(oracle.extrapolate(Z, X, 0.5), [[-0.5, 0.0], [-0.5, 0.0]], atol=1e-15)


@pytest.mark.parametrize("omega,c", [(0.5, 1.0), (1.0, 0.5), (2.0, 0.75)])
def test_constant_factors_are_a_single_omega(omega, c):
    D = _D(*synth.delaunay(40, seed=2))
    X0 = synth.initial_layout(40, 2, seed=2).astype(np.float64)
    ref = oracle.sor_run(D, X0, omega=omega * c, tol=1e-6, max_iter=40)
    got = oracle.sor_run(D, X0, omega=omega, tol=1e-6, max_iter=40, omega_vertex=np.full(40, c))
    assert got.iterations == ref.iterations
    assert got.trace_accept == ref.trace_accept
    assert np.allclose(got.trace_f, ref.trace_f, rtol=1e-11, atol=0)
    assert np.allclose(got.X, ref.X, rtol=0, atol=1e-9)


def test_zero_factors_are_algorithm_1():
    D = _D(*synth.grid(6, 6))
    X0 = synth.initial_layout(36, 2, seed=1).astype(np.float64)
    ref = oracle.sor_run(D, X0, omega=0.0, tol=1e-6, max_iter=50)
    got = oracle.sor_run(D, X0, omega=1.5, tol=1e-6, max_iter=50, omega_vertex=np.zeros(36))
    assert got.iterations == ref.iterations
    assert all(got.trace_accept)  # the candidate equals H(X^k): line 6 ties accept
    assert np.array_equal(got.X, ref.X)


def test_relabelling_equivariance():
    rp, ci = synth.delaunay(50, seed=3)
    n = len(rp) - 1
    D = _D(rp, ci)
    rng = np.random.default_rng(7)
    X0 = synth.initial_layout(n, 2, seed=3).astype(np.float64)
    m = rng.uniform(0.0, 2.0, n)
    perm = np.concatenate([[0], 1 + rng.permutation(n - 1)])  # new vertex a is old vertex perm[a]
    Dp = D[np.ix_(perm, perm)]
    a = oracle.sor_run(D, X0, omega=1.0, tol=1e-6, max_iter=30, omega_vertex=m)
    b = oracle.sor_run(Dp, X0[perm], omega=1.0, tol=1e-6, max_iter=30, omega_vertex=m[perm])
    assert a.iterations == b.iterations
    assert a.trace_accept == b.trace_accept
    assert np.allclose(a.trace_f, b.trace_f, rtol=1e-10, atol=0)
    assert np.allclose(a.X[perm], b.X, rtol=0, atol=1e-8)
    # a factor vector that is not relabelled gives a different run
    c = oracle.sor_run(Dp, X0[perm], omega=1.0, tol=1e-6, max_iter=30, omega_vertex=m)
    assert not np.allclose(c.trace_f[:5], b.trace_f[:5], rtol=1e-6, atol=0)


def test_acceptance_chain_with_factors():
    D = _D(*synth.delaunay(60, seed=4))
    X0 = synth.initial_layout(60, 2, seed=4).astype(np.float64)
    m = np.random.default_rng(4).uniform(0.0, 3.0, 60)
    for strategy in (oracle.OMEGA_FIXED, oracle.OMEGA_ENUM):
        r = oracle.sor_run(D, X0, omega=1.0, strategy=strategy, tol=1e-7, max_iter=40, omega_vertex=m)
        for k in range(r.iterations):
            assert r.trace_f[k + 1] <= r.trace_fH[k] + 1e-12   # line 6
            assert r.trace_fH[k] <= r.trace_f[k] * (1 + 1e-12)  # Prop. 2.2


def test_enumeration_with_unit_factors_is_the_scalar_enumeration():
    D = _D(*synth.grid(5, 6))
    X0 = synth.initial_layout(30, 2, seed=6).astype(np.float64)
    ref = oracle.sor_run(D, X0, strategy=oracle.OMEGA_ENUM, tol=1e-6, max_iter=20)
    got = oracle.sor_run(D, X0, strategy=oracle.OMEGA_ENUM, tol=1e-6, max_iter=20, omega_vertex=np.ones(30))
    assert got.trace_omega == ref.trace_omega
    assert np.allclose(got.trace_f, ref.trace_f, rtol=1e-11, atol=0)
