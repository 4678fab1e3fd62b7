"""Per-vertex relaxation factors (Sec. 6: omega_i per vertex, here
omega_i = omega m_i) through the C ABI, against the FP64 oracle.

Tolerances as for the single-omega runs: one step 1e-4 relative on the
layout (CG to relative residual 1e-6), converged runs 1e-4 relative on the
final stress and iterations within 2 % (at least 1).
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


def _D(rp, ci):
    st, D = oracle.apsp(rp, ci, policy=1)
    return D


def _factors(n, seed, hi=2.0):
    return np.random.default_rng(seed).uniform(0.0, hi, n).astype(np.float32)


@pytest.mark.parametrize("graph,dim,omega", [(lambda: synth.delaunay(1000, seed=3), 2, 1.0),
                                             (lambda: synth.erdos_renyi(300, 4.0, seed=1), 3, 0.5),
                                             (lambda: synth.random_binary_tree(383, seed=2), 1, 1.5)])
def test_one_step_matches_oracle(graph, dim, omega):
    rp, ci = graph()
    n = len(rp) - 1
    D = _D(rp, ci)
    X0 = synth.initial_layout(n, dim, seed=5)
    m = _factors(n, 11)
    Xn, fn, acc, _, _ = oracle.sor_step(X0.astype(np.float64), D, omega, omega_vertex=m.astype(np.float64))
    X = X0.copy()
    with api.Layout(rp, ci, dim=dim, disconnected_policy=1) as L:
        L.set_vertex_omega(m)
        f, accepted, crit = L.sor_step(X, k=0, omega=omega, cg_tol=1e-6, cg_max=500)
    assert accepted == acc
    assert np.linalg.norm(X - Xn) <= 1e-4 * np.linalg.norm(Xn)
    assert f == pytest.approx(fn, rel=1e-4)


def test_converged_run_grid20_matches_oracle():
    rp, ci = synth.grid(20, 20)
    D = _D(rp, ci)
    X0 = synth.initial_layout(400, 2, seed=0)
    m = _factors(400, 3)
    ref = oracle.sor_run(D, X0.astype(np.float64), omega=1.0, tol=1e-4, max_iter=1000,
                         omega_vertex=m.astype(np.float64))
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        L.set_vertex_omega(m)
        r = L.run(X, trace=True, omega=1.0, tol=1e-4, max_iter=1000)
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert abs(r.iterations - ref.iterations) <= max(1, math.ceil(0.02 * ref.iterations))
    k = min(5, r.iterations)
    assert np.array_equal(r.accepted[:k].astype(bool), np.array(ref.trace_accept[:k]))
    assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])


def test_enumeration_with_factors_matches_oracle():
    rp, ci = synth.grid(10, 10)
    D = _D(rp, ci)
    X0 = synth.initial_layout(100, 2, seed=4)
    m = _factors(100, 5, hi=1.5)
    ref = oracle.sor_run(D, X0.astype(np.float64), strategy=oracle.OMEGA_ENUM, tol=1e-4, max_iter=60,
                         omega_vertex=m.astype(np.float64))
    X = X0.copy()
    with api.Layout(rp, ci, dim=2) as L:
        L.set_vertex_omega(m)
        r = L.run(X, trace=True, strategy=api.OMEGA_ENUM, tol=1e-4, max_iter=60)
    k = min(5, r.iterations, ref.iterations)
    assert np.array_equal(r.omega[:k], np.array(ref.trace_omega[:k]))
    assert r.stress == pytest.approx(ref.stress, rel=1e-4)
    assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])


def test_unit_and_cleared_factors_equal_a_single_omega():
    import torch
    rp, ci = synth.delaunay(700, seed=9)
    n = len(rp) - 1
    X0 = synth.initial_layout(n, 2, seed=9)
    with api.Layout(rp, ci, dim=2) as L:
        Xa = X0.copy()
        ra = L.run(Xa, omega=0.5, tol=1e-4, max_iter=300)
        L.set_vertex_omega(torch.ones(n, dtype=torch.float32, device="cuda"))
        Xb = X0.copy()
        rb = L.run(Xb, omega=0.5, tol=1e-4, max_iter=300)
        L.set_vertex_omega(None)
        Xc = X0.copy()
        rc = L.run(Xc, omega=0.5, tol=1e-4, max_iter=300)
    for r in (rb, rc):
        assert r.stress == pytest.approx(ra.stress, rel=1e-5)
        assert abs(r.iterations - ra.iterations) <= max(1, math.ceil(0.02 * ra.iterations))


def test_bad_factors_are_rejected():
    rp, ci = synth.grid(4, 4)
    with api.Layout(rp, ci, dim=2) as L:
        for bad in (np.full(16, -1.0, np.float32), np.array([np.nan] + [1.0] * 15, np.float32)):
            with pytest.raises(api.FdError) as e:
                L.set_vertex_omega(bad)
            assert e.value.status == 1  # FD_ERR_ARG
        with pytest.raises(ValueError):
            L.set_vertex_omega(np.ones(15, np.float32))
