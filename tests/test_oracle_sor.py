"""Pins of the oracle's majorization step H (Eq. (4), Eq. (2-5)) and of
Algorithms 1 and 2 (Sec. 4), with the omega strategies of Sec. 5.2.

Pins: the residual of Eq. (2-5) and the pinning x_1 = 0; the Moore-Penrose
solution (a different method); H minimises g(., X) (Eq. (4)); the chain of
Prop. 2.2; analytic optima of small graphs; the linear rate 1 - lambda_min of
Theorem 3.2; the SplitMix64 test vector and the prior of Sec. 5.2.3.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import synth


def _D(rp, ci):
    st, D = oracle.apsp(rp, ci, policy=1)
    return D


def test_pinned_solve_residual_and_pseudoinverse():
    D = _D(*synth.delaunay(60, seed=1))
    X = np.random.default_rng(1).random((60, 2))
    b = oracle.rhs(X, D)
    Z = oracle.PinnedSolver(D).solve(b)
    assert np.all(Z[0] == 0.0)
    L = oracle.lw_dense(D)
    assert np.abs(L @ Z - b).max() <= 1e-11 * np.abs(b).max()
    # the Moore-Penrose solution differs only by a translation
    Zp = np.linalg.pinv(L) @ b
    assert np.allclose(Zp - Zp[0], Z, rtol=1e-9, atol=1e-11)


def test_H_minimises_majorant():
    D = _D(*synth.erdos_renyi(20, 4.0, seed=2))
    rng = np.random.default_rng(2)
    X = rng.random((20, 2))
    Z = oracle.H(X, D)
    g0 = oracle.majorant(Z, X, D)
    for _ in range(8):
        V = rng.standard_normal((20, 2)) * 1e-2
        assert oracle.majorant(Z + V, X, D) >= g0 - 1e-12


def test_majorization_chain():
    # Prop. 2.2: f(X^{k+1}) <= g(X^{k+1}, X^k) <= g(X^k, X^k) = f(X^k).
    D = _D(*synth.random_binary_tree(25, seed=3))
    X = np.random.default_rng(3).random((25, 2))
    for _ in range(5):
        Z = oracle.H(X, D)
        fZ, gZ, fX = oracle.stress(Z, D), oracle.majorant(Z, X, D), oracle.stress(X, D)
        assert fZ <= gZ + 1e-12 and gZ <= fX + 1e-12
        X = Z


def test_K2_one_step_exact():
    D = _D(*synth.path(2))
    X = np.array([[0.2, 0.7], [0.9, 0.1]])
    Z = oracle.H(X, D)
    assert np.linalg.norm(Z[1] - Z[0]) == pytest.approx(1.0, abs=1e-14)
    assert oracle.stress(Z, D) == pytest.approx(0.0, abs=1e-28)


def test_algorithm1_monotone_and_omega0_identity():
    D = _D(*synth.grid(6, 6))
    X0 = synth.initial_layout(36, 2, seed=0).astype(np.float64)
    r = oracle.sor_run(D, X0, omega=0.0, tol=1e-6, max_iter=60)
    f = np.array(r.trace_f)
    assert np.all(np.diff(f) <= 1e-12 * f[:-1])
    # omega = 0 is Algorithm 1: the iterates are plain repeated H steps
    X = X0.copy()
    solver = oracle.PinnedSolver(D)
    for k in range(r.iterations):
        X = oracle.H(X, D, solver)
    assert np.array_equal(X, r.X)


def test_algorithm2_acceptance_chain():
    D = _D(*synth.delaunay(50, seed=5))
    X0 = synth.initial_layout(50, 2, seed=5).astype(np.float64)
    for om in (0.5, 1.5, 3.0):
        r = oracle.sor_run(D, X0, omega=om, tol=1e-7, max_iter=80)
        for k in range(r.iterations):
            # accepted stress never exceeds f(H(X^k)) <= f(X^k) (line 6, Prop. 2.2)
            assert r.trace_f[k + 1] <= r.trace_fH[k] + 1e-12
            assert r.trace_fH[k] <= r.trace_f[k] * (1 + 1e-12)


def _relaxed_run(D, X0, **kw):
    return oracle.sor_run(D, X0, tol=1e-12, max_iter=400, **kw)


def test_square_optimum():
    # C4: square of side s* = (8 + 2 sqrt 2)/10 minimises 4(s-1)^2 + (sqrt2 s - 2)^2/2.
    D = _D(*synth.cycle(4))
    s_star = (8 + 2 * math.sqrt(2)) / 10
    f_star = 4 * (s_star - 1) ** 2 + 0.5 * (math.sqrt(2) * s_star - 2) ** 2
    X0 = np.array([[0.0, 0.0], [1.0, 0.1], [1.1, 0.9], [0.05, 1.0]])
    for om in (0.0, 0.5):
        r = _relaxed_run(D, X0, omega=om)
        assert r.stress == pytest.approx(f_star, rel=1e-9)
        side = [np.linalg.norm(r.X[i] - r.X[(i + 1) % 4]) for i in range(4)]
        assert np.allclose(side, s_star, rtol=1e-6)


def test_star_optimum():
    D = _D(*synth.star(3))
    r_star = (6 + 3 * math.sqrt(3)) / 10.5
    f_star = 3 * (r_star - 1) ** 2 + 0.75 * (math.sqrt(3) * r_star - 2) ** 2
    X0 = np.array([[0.0, 0.0], [1.0, 0.1], [-0.4, 0.8], [-0.5, -0.9]])
    r = _relaxed_run(D, X0, omega=0.5)
    assert r.stress == pytest.approx(f_star, rel=1e-9)
    rad = np.linalg.norm(r.X[1:] - r.X[0], axis=1)
    assert np.allclose(rad, r_star, rtol=1e-6)


def _hessian_fd(D, x, h=1e-5):
    # Hessian of f by central differences of the force F = -1/2 grad f,
    # in the flattened ordering (vertex, coordinate).
    n, dim = x.shape
    Hm = np.zeros((n * dim, n * dim))
    for i in range(n):
        for c in range(dim):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            Hm[:, i * dim + c] = (-2.0 * oracle.forces(xp, D) + 2.0 * oracle.forces(xm, D)).ravel() / (2 * h)
    return 0.5 * (Hm + Hm.T)


def _theorem_3_2(D, X0, pert, nsteps=30, amp=1e-4):
    import scipy.linalg as sla
    n, dim = X0.shape
    r = oracle.sor_run(D, X0, omega=0.0, tol=1e-15, max_iter=4000)
    xs = r.X
    Hf = _hessian_fd(D, xs)[dim:, dim:]                              # D^2 f, vertex 1 pinned
    G = np.kron(2.0 * oracle.lw_dense(D), np.eye(dim))[dim:, dim:]   # D_11 g = 2 L^W per coordinate
    lam = sla.eigh(Hf, G, eigvals_only=True)
    solver = oracle.PinnedSolver(D)
    x = xs + amp * pert
    x[0] = 0.0
    steps = []
    for _ in range(nsteps):
        xn = oracle.H(x, D, solver)
        steps.append(np.linalg.norm(xn - x))
        x = xn
    # Jacobian of H at x* by central differences, pinned coordinates
    h = 1e-6
    J = np.zeros((n * dim, n * dim))
    for i in range(n):
        for c in range(dim):
            xp, xm = xs.copy(), xs.copy()
            xp[i, c] += h
            xm[i, c] -= h
            J[:, i * dim + c] = (oracle.H(xp, D, solver) - oracle.H(xm, D, solver)).ravel() / (2 * h)
    return lam, np.array(steps), J[dim:, dim:]


def test_theorem_3_2_rate_d2():
    # Theorem 3.2: H'(x*) = I - [D_11 g]^-1 D^2 f (Eq. (8)-(9)), so Algorithm 1
    # converges linearly at rate 1 - lambda_min of D^2 f z = lambda D_11 g z.
    # In d = 2 a rigid rotation about the pinned vertex is neutral (lambda = 0,
    # H' eigenvalue 1, no step along it) and is left out of the rate.
    D = _D(*synth.delaunay(9, seed=4))
    X0 = synth.initial_layout(9, 2, seed=4).astype(np.float64)
    pert = np.random.default_rng(0).standard_normal((9, 2))
    lam, steps, J = _theorem_3_2(D, X0, pert, nsteps=110, amp=1e-3)
    assert abs(lam[0]) < 1e-5 and lam[1] > 1e-2      # one rotation mode, then a gap
    assert lam.max() <= 1.0 + 1e-6                   # g majorises f: D_11 g >= D^2 f
    ev = np.sort(np.linalg.eigvals(J).real)
    assert np.allclose(ev, np.sort(1.0 - lam), atol=1e-5)
    rate = 1.0 - lam[1]
    ratios = steps[90:110] / steps[89:109]
    assert ratios.mean() == pytest.approx(rate, abs=1e-3)


def test_theorem_3_2_d1_is_one_step():
    # In d = 1, away from coincident vertices ||x_i - x_j|| is locally linear,
    # so D^2 f = D_11 g: every lambda is 1 and the rate 1 - lambda is 0.
    D = _D(*synth.cycle(5))
    x0 = np.array([[0.0], [0.9], [2.1], [1.2], [-0.3]])
    lam, steps, J = _theorem_3_2(D, x0, np.array([[0.0], [0.3], [-0.5], [0.2], [0.7]]))
    assert np.allclose(lam, 1.0, atol=1e-4)
    assert np.allclose(J, 0.0, atol=1e-6)
    assert steps[1] <= 1e-12 * max(steps[0], 1e-300) + 1e-15


def test_splitmix64_vector_and_prior():
    # SplitMix64, seed 1234567: first outputs of the published reference generator.
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [oracle.splitmix64(1234567, k) for k in range(5)] == expect
    draws = np.array([oracle.omega_draw(11, k) for k in range(40000)])
    for om, p in zip((0.5, 1.0, 1.5, 2.0), (0.3, 0.3, 0.2, 0.2)):
        freq = np.mean(draws == om)
        assert abs(freq - p) < 4 * math.sqrt(p * (1 - p) / len(draws))


def test_enumerate_strategy_is_argmin():
    D = _D(*synth.grid(5, 5))
    X = synth.initial_layout(25, 2, seed=2).astype(np.float64)
    solver = oracle.PinnedSolver(D)
    Xn, fn, acc, om, fZ = oracle.sor_step(X, D, 0.0, oracle.OMEGA_ENUM, solver)
    Z = oracle.H(X, D, solver)
    fs = [oracle.stress((1 + w) * Z - w * X, D) for w in np.arange(0, 9.01, 0.5)]
    assert fn == pytest.approx(min(fs), rel=1e-15)
    assert om == 0.5 * int(np.argmin(fs))
    assert fn <= fZ


# ---------------------------------------------------------------------------
# The termination criterion.  The paper leaves the rule open ("until some
# termination conditions were satisfied", Algorithms 1 and 2; Table 1 quotes a
# relative error per data set); the library's two readings are the relative
# displacement of centred layouts and the relative decrease of the stress.
# Pins: values worked by hand, the invariances a displacement measure of
# layouts defined up to a similarity must have, the linear rate of
# Theorem 3.2 that the displacement inherits, and the run's bookkeeping
# (which layouts and stresses enter).  A criterion without centring, divided
# by the old layout's norm or fed the un-accepted stress fails one of them.
# ---------------------------------------------------------------------------

def test_criterion_rel_disp_by_hand():
    # two vertices: (0,0),(2,0) -> (1,0),(2,0).  Centred: (-1,0),(1,0) and
    # (-0.5,0),(0.5,0); displacement sqrt(0.5) over sqrt(0.5) = 1.
    # (without centring: 1/sqrt(5); divided by the old norm: 0.5)
    Xo = np.array([[0.0, 0.0], [2.0, 0.0]])
    Xn = np.array([[1.0, 0.0], [2.0, 0.0]])
    assert oracle.criterion(oracle.STOP_REL_DISP, Xo, Xn, 0.0, 0.0) == pytest.approx(1.0, rel=1e-15)
    # a path of three: (0,0),(1,0),(2,0) -> (0,0),(1,1),(2,0).  Means (1,0) and
    # (1,1/3); the centred difference is (0,-1/3),(0,2/3),(0,-1/3), squared norm
    # 2/3; the centred new layout has squared norm 8/3; sqrt(1/4) = 1/2.
    Xo = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    Xn = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 0.0]])
    assert oracle.criterion(oracle.STOP_REL_DISP, Xo, Xn, 0.0, 0.0) == pytest.approx(0.5, rel=1e-15)
    # a layout collapsed to one point has nothing left to move: 0
    assert oracle.criterion(oracle.STOP_REL_DISP, Xo, np.ones((3, 2)), 0.0, 0.0) == 0.0


def test_criterion_rel_stress_by_hand():
    # (f_k - f_{k+1}) / f_k: 4 -> 3 gives 1/4 (divided by the new stress: 1/3)
    assert oracle.criterion(oracle.STOP_REL_STRESS, None, None, 4.0, 3.0) == 0.25
    assert oracle.criterion(oracle.STOP_REL_STRESS, None, None, 0.0, 0.0) == 0.0
    with pytest.raises(ValueError):
        oracle.criterion(7, None, None, 1.0, 1.0)


def test_criterion_rel_disp_invariances():
    # the layouts are defined up to translation (the pinning of Sec. 2 moves
    # them every H step), so the measure ignores a separate translation of
    # each; a common rotation or scaling of both leaves it unchanged too
    rng = np.random.default_rng(5)
    Xo = rng.random((17, 2))
    Xn = Xo + 0.05 * rng.standard_normal((17, 2))
    c0 = oracle.criterion(oracle.STOP_REL_DISP, Xo, Xn, 0.0, 0.0)
    c1 = oracle.criterion(oracle.STOP_REL_DISP, Xo + np.array([3.0, -1.0]), Xn + np.array([-7.0, 2.5]), 0.0, 0.0)
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    c2 = oracle.criterion(oracle.STOP_REL_DISP, Xo @ Q.T, Xn @ Q.T, 0.0, 0.0)
    c3 = oracle.criterion(oracle.STOP_REL_DISP, 4.0 * Xo, 4.0 * Xn, 0.0, 0.0)
    assert c1 == pytest.approx(c0, rel=1e-12)
    assert c2 == pytest.approx(c0, rel=1e-12)
    assert c3 == pytest.approx(c0, rel=1e-12)
    # but not under a change of one layout's scale alone
    assert abs(oracle.criterion(oracle.STOP_REL_DISP, Xo, 2.0 * Xn, 0.0, 0.0) - c0) > 0.1


def test_criterion_run_bookkeeping():
    # sor_run measures each iteration between consecutive accepted layouts
    # (REL_DISP) and between consecutive accepted stresses (REL_STRESS), and
    # stops at the first iteration whose criterion is below tol
    D = _D(*synth.delaunay(40, seed=8))
    X0 = synth.initial_layout(40, 2, seed=8).astype(np.float64)
    solver = oracle.PinnedSolver(D)
    r = oracle.sor_run(D, X0, omega=1.0, tol=0.0, max_iter=12, solver=solver)
    rs = oracle.sor_run(D, X0, omega=1.0, tol=0.0, max_iter=12, solver=solver, stop=oracle.STOP_REL_STRESS)
    X, f = X0.copy(), oracle.stress(X0, D)
    saw_accept_below_h = False
    for k in range(12):
        Xn, fn, acc, _, fZ = oracle.sor_step(X, D, 1.0, oracle.OMEGA_FIXED, solver)
        assert r.trace_crit[k] == oracle.criterion(oracle.STOP_REL_DISP, X, Xn, f, fn)
        assert rs.trace_crit[k] == (f - fn) / f
        saw_accept_below_h |= acc and fn < fZ
        X, f = Xn, fn
    assert saw_accept_below_h  # the accepted stress, not f(H(X^k)), enters REL_STRESS
    tol = 0.5 * (r.trace_crit[5] + r.trace_crit[6])
    first = next(k for k, c in enumerate(r.trace_crit) if c < tol)
    r2 = oracle.sor_run(D, X0, omega=1.0, tol=tol, max_iter=12, solver=solver)
    assert r2.iterations == first + 1 and r2.converged


def test_criterion_decays_at_theorem_3_2_rate():
    # Algorithm 1 near x*: X^{k+1} - X^k shrinks by 1 - lambda_min per step
    # (Theorem 3.2), and the centred norm of X^{k+1} tends to that of x*, so
    # the REL_DISP criterion decays at the same rate
    D = _D(*synth.delaunay(9, seed=4))
    X0 = synth.initial_layout(9, 2, seed=4).astype(np.float64)
    pert = np.random.default_rng(0).standard_normal((9, 2))
    lam, steps, J = _theorem_3_2(D, X0, pert, nsteps=2, amp=1e-3)
    rate = 1.0 - lam[1]
    xs = oracle.sor_run(D, X0, omega=0.0, tol=1e-15, max_iter=4000).X
    r = oracle.sor_run(D, xs + 1e-3 * pert, omega=0.0, tol=0.0, max_iter=110)
    c = np.array(r.trace_crit)
    assert (c[91:110] / c[90:109]).mean() == pytest.approx(rate, abs=1e-3)
