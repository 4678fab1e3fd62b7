"""FP64 CPU oracle for the SOR stress-majorization layout method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in ``paper_1711_01228_gb300``
and imports nothing from it; the only common inputs are arrays made by the
seeded generators in ``paper_1711_01228_gb300.synth``, which hold none of the
method's arithmetic.

Paper: Wang & Wang, "A Fast Successive Over-Relaxation Algorithm for
Force-Directed Network Graph Drawing", Sci. China Inf. Sci. 55:677 (2012).

What each function follows, and what pins it (the tests under ``tests/`` named
``test_oracle_*`` hold the pins):

=====================  ====================================  ===============================================
function               paper passage                          pin
=====================  ====================================  ===============================================
apsp / bfs_row         d_ij "predefined ideal distance",       scipy.sparse.csgraph.shortest_path; Manhattan
                       Sec. 2 Eq. (1); shortest paths as in    distance on grids; Floyd-Warshall brute force
                       Gansner et al. (Sec. 2, Prop. 2.3)
stress                 Eq. (1), w_ij = d_ij^-2 (Sec. 5.1)     closed forms on 2-4 vertex graphs; trace form
                                                              g(X,X) of Prop. 2.1; invariances
rhs  (L^X X)           Prop. 2.1, Eq. (2-5)                   finite-difference gradient of sum w d r
lw_matvec (L^W P)      Prop. 2.1                              finite-difference gradient of sum w r^2; L^W 1=0
forces                 -1/2 grad of Eq. (1)                   finite differences of stress
PinnedSolver (H)       Eq. (4), Eq. (2-5), pinning x_1 = 0    residual of Eq. (2-5); majorization chain of
                       (Sec. 2 after Prop. 2.3)               Prop. 2.2; H minimises g(., X); K2 one-step
sor_run                Algorithm 1 (omega = 0), Algorithm 2,  monotone stress (Prop. 2.2); omega=0 equals
                       Eq. (10); strategies of Sec. 5.2       Algorithm 1; analytic optima (C4, K1,3);
                                                              observed rate = 1 - lambda_min (Thm 3.2)
omega_draw             probabilistic strategy, Sec. 5.2.3     splitmix64 published test vector; prior
                                                              frequencies
shifted_inverse        solver of Eq. (2-5) with L^W fixed        closed forms on K2 and K5; A'^-1 1 = 1/sigma;
                       (Sec. 2): inverse of L^W + sigma/n 11^T  A'^-1 b minus the pinned Cholesky solve is a
                                                              translation (zero-sum b)
extrapolate            line 5 of Algorithm 2, Eq. (10); the   m = 1 and m = c reduce to Eq. (10) with omega
                       per-vertex omega_i of Sec. 6           and omega c; m = 0 gives Algorithm 1; candidate
                                                              derived by hand on K2; relabelling equivariance
criterion              termination of Algorithms 1 and 2      values worked by hand (two vertices, a path of
                       (the library's reading, below)         three, 4 -> 3); invariance under separate
                                                              translations and common rotation / scaling; the
                                                              REL_DISP sequence decays at the rate 1 -
                                                              lambda_min of Thm 3.2; sor_run's bookkeeping
force_abs /            sum_j |term| of the rows of -1/2 grad  = |F| with one term (K2) and for a row of one
force_row_abs          of Eq. (1) (a tolerance scale)         sign; >= |F| (triangle inequality), strictly for
                                                              mixed signs
stress_stream          Eq. (1), rows streamed by BFS          equals `stress` on a stored D; a split over
                                                              processes equals the serial sum to rounding
=====================  ====================================  ===============================================

The termination rule is not defined by the paper ("until some termination
conditions were satisfied", Algorithms 1 and 2; Table 1 quotes a relative
error per data set); the two rules here are the library's readings (relative
displacement of centred layouts, or relative stress decrease).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

ERR_DISCONNECTED = 3

STOP_REL_DISP = 0
STOP_REL_STRESS = 1
OMEGA_FIXED = 0
OMEGA_PROB = 1
OMEGA_ENUM = 2

_lib_handle = None


def build() -> str:
    """Compile fd_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32 = ctypes.c_int
        lib.orc_bfs.argtypes = [i32, P, P, i32, P, P]
        lib.orc_apsp.argtypes = [i32, P, P, P, i32, P]
        lib.orc_apsp.restype = i32
        lib.orc_stress.argtypes = [i32, i32, P, P]
        lib.orc_stress.restype = ctypes.c_double
        for name in ("orc_rhs", "orc_lw_matvec", "orc_forces"):
            getattr(lib, name).argtypes = [i32, i32, P, P, P]
        lib.orc_force_row.argtypes = [i32, i32, P, i32, P, P]
        lib.orc_rhs_row.argtypes = [i32, i32, P, i32, P, P]
        lib.orc_stress_stream.argtypes = [i32, i32, P, P, P, ctypes.c_double, ctypes.POINTER(i32)]
        lib.orc_stress_stream.restype = ctypes.c_double
        lib.orc_stress_stream_rows.argtypes = [i32, i32, P, P, P, ctypes.c_double, i32, i32, ctypes.POINTER(i32)]
        lib.orc_stress_stream_rows.restype = ctypes.c_double
        lib.orc_force_row_abs.argtypes = [i32, i32, P, i32, P, P]
        lib.orc_stress_stream_rows_multi.argtypes = [i32, i32, P, P, P, P, ctypes.c_double, i32, i32, P,
                                                     ctypes.POINTER(i32)]
        _lib_handle = lib
    return _lib_handle


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(X) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(X, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# --------------------------------------------------------------------------
# Ideal distances
# --------------------------------------------------------------------------

def apsp(row_ptr, col_idx, edge_len=None, policy: int = 0):
    """Dense [n, n] FP64 matrix of ideal distances d_ij (shortest paths).

    Returns (status, D); status 3 means a disconnected graph under policy 0.
    Policy 1 gives unreachable pairs d = (largest finite d) + 1.
    """
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = rp.shape[0] - 1
    D = np.zeros((n, n), dtype=np.float64)
    ln = None if edge_len is None else _f64(edge_len)
    st = _lib().orc_apsp(n, _p(rp), _p(ci), None if ln is None else _p(ln), int(policy), _p(D))
    return int(st), D


def bfs_row(row_ptr, col_idx, src: int) -> np.ndarray:
    """Hop distances from one source (int32, -1 if unreachable)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = rp.shape[0] - 1
    dist = np.empty(n, dtype=np.int32)
    q = np.empty(n, dtype=np.int32)
    _lib().orc_bfs(n, _p(rp), _p(ci), int(src), _p(dist), _p(q))
    return dist


# --------------------------------------------------------------------------
# Pair functions (Eq. (1), Prop. 2.1)
# --------------------------------------------------------------------------

def stress(X, D) -> float:
    """f(X) of Eq. (1) with w = d^-2."""
    X, D = _f64(X), _f64(D)
    n, dim = X.shape
    return float(_lib().orc_stress(n, dim, _p(X), _p(D)))


def _pairfn(name, X, D):
    X, D = _f64(X), _f64(D)
    n, dim = X.shape
    out = np.zeros_like(X)
    getattr(_lib(), name)(n, dim, _p(X), _p(D), _p(out))
    return out


def rhs(X, D) -> np.ndarray:
    """b = L^X X, the right-hand side of Eq. (2-5)."""
    return _pairfn("orc_rhs", X, D)


def lw_matvec(P, D) -> np.ndarray:
    """L^W P."""
    return _pairfn("orc_lw_matvec", P, D)


def forces(X, D) -> np.ndarray:
    """F = (L^X - L^W) X = -1/2 grad f(X)."""
    return _pairfn("orc_forces", X, D)


def force_row(X, i: int, drow) -> np.ndarray:
    X, dr = _f64(X), _f64(drow)
    n, dim = X.shape
    out = np.zeros(dim)
    _lib().orc_force_row(n, dim, _p(X), int(i), _p(dr), _p(out))
    return out


def force_row_abs(X, i: int, drow) -> np.ndarray:
    """Per coordinate c, A_ic = sum_j |w_ij (d_ij / r_ij - 1)(x_ic - x_jc)|: the
    magnitude of the terms that make up F_ic (|F_ic| <= A_ic).  Rounding in
    any summation of the row is bounded relative to A_ic, so per-element force
    tolerances are stated against it."""
    X, dr = _f64(X), _f64(drow)
    n, dim = X.shape
    out = np.zeros(dim)
    _lib().orc_force_row_abs(n, dim, _p(X), int(i), _p(dr), _p(out))
    return out


def force_abs(X, D) -> np.ndarray:
    """force_row_abs for every row of a dense D: [n, dim]."""
    X, D = _f64(X), _f64(D)
    return np.stack([force_row_abs(X, i, D[i]) for i in range(X.shape[0])])


def rhs_row(X, i: int, drow) -> np.ndarray:
    X, dr = _f64(X), _f64(drow)
    n, dim = X.shape
    out = np.zeros(dim)
    _lib().orc_rhs_row(n, dim, _p(X), int(i), _p(dr), _p(out))
    return out


def _stress_rows(X, rp, ci, dfill, i0, i1) -> float:
    n, dim = X.shape
    st = ctypes.c_int(0)
    f = _lib().orc_stress_stream_rows(n, dim, _p(X), _p(rp), _p(ci), float(dfill), int(i0), int(i1),
                                      ctypes.byref(st))
    if st.value != 0:
        raise ValueError(f"stress_stream status {st.value}")
    return float(f)


_POOL_ARGS = None


def _pool_init(*args):
    global _POOL_ARGS
    _POOL_ARGS = args


def _stress_rows_task(rng):
    X, rp, ci, dfill = _POOL_ARGS
    return _stress_rows(X, rp, ci, dfill, rng[0], rng[1])


def _row_ranges(n, workers):
    cuts = np.linspace(0, n, 8 * workers + 1).astype(int)
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def _stress_rows_multi(Xs, rp, ci, dfill, i0, i1) -> np.ndarray:
    Xs = [_f64(X) for X in Xs]
    n = Xs[0].shape[0]
    dims = np.array([X.shape[1] for X in Xs], dtype=np.int32)
    ptrs = (ctypes.c_void_p * len(Xs))(*[X.ctypes.data for X in Xs])
    out = np.zeros(len(Xs))
    st = ctypes.c_int(0)
    _lib().orc_stress_stream_rows_multi(n, len(Xs), _p(dims), ptrs, _p(rp), _p(ci), float(dfill), int(i0), int(i1),
                                        _p(out), ctypes.byref(st))
    if st.value != 0:
        raise ValueError(f"stress_stream status {st.value}")
    return out


def _stress_rows_multi_task(rng):
    Xs, rp, ci, dfill = _POOL_ARGS
    return _stress_rows_multi(Xs, rp, ci, dfill, rng[0], rng[1])


def stress_stream_multi(Xs, row_ptr, col_idx, dfill: float = -1.0, workers: int = 1) -> np.ndarray:
    """stress_stream of several layouts of one graph (any dimensions), one BFS
    per row for all of them; rows split over `workers` spawned processes as
    in stress_stream."""
    Xs = [_f64(X) for X in Xs]
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = Xs[0].shape[0]
    if workers <= 1 or n < 4096:
        return _stress_rows_multi(Xs, rp, ci, dfill, 0, n)
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(Xs, rp, ci, float(dfill))) as pool:
        parts = pool.map(_stress_rows_multi_task, _row_ranges(n, workers), chunksize=1)
    return np.sum(parts, axis=0)


def stress_stream(X, row_ptr, col_idx, dfill: float = -1.0, workers: int = 1) -> float:
    """Eq. (1) for unit-edge graphs, one BFS per row instead of a stored D.

    Eq. (1) sums over the rows i of sum_{j > i}; with workers > 1 the rows are
    split into ranges evaluated by that many processes (started with the
    'spawn' method, so that a process holding a GPU context can call this)
    and the parts are added (only the order of the FP64 additions differs)."""
    X = _f64(X)
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = X.shape[0]
    if workers <= 1 or n < 4096:
        return _stress_rows(X, rp, ci, dfill, 0, n)
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(X, rp, ci, float(dfill))) as pool:
        parts = pool.map(_stress_rows_task, _row_ranges(n, workers), chunksize=1)
    return float(sum(parts))


# --------------------------------------------------------------------------
# Matrices of Prop. 2.1 (explicit, for small n) and the majorant g
# --------------------------------------------------------------------------

def weights(D) -> np.ndarray:
    """w_ij = d_ij^-2 off the diagonal, 0 on it (Sec. 5.1)."""
    D = _f64(D)
    W = np.zeros_like(D)
    off = ~np.eye(D.shape[0], dtype=bool)
    W[off] = 1.0 / (D[off] ** 2)
    return W


def lw_dense(D) -> np.ndarray:
    """L^W of Prop. 2.1 as a dense matrix."""
    W = weights(D)
    L = -W
    np.fill_diagonal(L, W.sum(axis=1))
    return L


def ly_dense(Y, D) -> np.ndarray:
    """L^Y of Prop. 2.1 as a dense matrix (entries 0 where y_i = y_j)."""
    Y, D = _f64(Y), _f64(D)
    n = Y.shape[0]
    L = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            r = float(np.sqrt(np.sum((Y[i] - Y[j]) ** 2)))
            if r != 0.0:
                L[i, j] = -(1.0 / D[i, j] ** 2) * D[i, j] / r
    np.fill_diagonal(L, -L.sum(axis=1))
    return L


def majorant(X, Y, D) -> float:
    """g(X, Y) = tr(X^T L^W X) - 2 tr(X^T L^Y Y) + C of Eq. (2)."""
    X, Y, D = _f64(X), _f64(Y), _f64(D)
    iu = np.triu_indices(D.shape[0], 1)
    C = float(np.sum((1.0 / D[iu] ** 2) * D[iu] ** 2))
    return float(np.trace(X.T @ lw_dense(D) @ X) - 2.0 * np.trace(X.T @ ly_dense(Y, D) @ Y) + C)


# --------------------------------------------------------------------------
# The majorization step H (Eq. (4), Eq. (2-5)) with the pinning x_1 = 0
# --------------------------------------------------------------------------

class PinnedSolver:
    """Solves L^W Z = b with the first vertex pinned at the origin.

    The paper removes the first row and column of L^W and the first row of
    the right-hand side; the reduced matrix is strictly diagonally dominant
    and positive definite, and is factored here once by dense Cholesky
    (one of the solvers the paper names after Prop. 2.3).
    """

    def __init__(self, D):
        D = _f64(D)
        self.n = D.shape[0]
        if self.n > 1:
            A = lw_dense(D)[1:, 1:]
            self.L = np.linalg.cholesky(A)
        else:
            self.L = None

    def solve(self, b) -> np.ndarray:
        b = _f64(b)
        Z = np.zeros_like(b)
        if self.n <= 1:
            return Z
        import scipy.linalg as sla
        y = sla.solve_triangular(self.L, b[1:], lower=True)
        Z[1:] = sla.solve_triangular(self.L.T, y, lower=False)
        return Z


def shifted_inverse(D) -> np.ndarray:
    """Dense inverse of A' = L^W + (sigma / n) 1 1^T, sigma = mean_i s_i.

    L^W is singular with null vector 1 (Prop. 2.1); the shift gives 1 the
    eigenvalue sigma and leaves the rest of the spectrum, so A' is positive
    definite.  For a right-hand side b with zero sum, A'^-1 b solves
    L^W z = b (the solution of zero sum), which differs from the pinned
    solution of Eq. (2-5) by a translation.  The direct solver of the
    library applies this matrix in every H step.
    """
    L = lw_dense(D)
    n = L.shape[0]
    sigma = float(np.trace(L)) / n if n else 1.0
    if not sigma > 0.0:
        sigma = 1.0  # n = 1
    return np.linalg.inv(L + sigma / n)


def H(X, D, solver: PinnedSolver | None = None) -> np.ndarray:
    """X^{k+1} = H(X^k): argmin_X g(X, X^k), Eq. (4)."""
    solver = solver or PinnedSolver(D)
    return solver.solve(rhs(X, D))


# --------------------------------------------------------------------------
# Relaxation factors (Sec. 5.2)
# --------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, k: int) -> int:
    """k-th output (k = 0, 1, ...) of SplitMix64 seeded with `seed`
    (Steele, Lea & Flood, OOPSLA 2014; constants of Vigna's splitmix64.c)."""
    z = (seed + (k + 1) * _GAMMA) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


PROB_OMEGAS = (0.5, 1.0, 1.5, 2.0)
PROB_CUMULATIVE = (0.3, 0.6, 0.8, 1.0)


def omega_draw(seed: int, k: int) -> float:
    """Probabilistic strategy (Sec. 5.2.3): one roulette draw per iteration
    from the prior P(0.5)=P(1.0)=0.3, P(1.5)=P(2.0)=0.2."""
    u = (splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)
    for om, c in zip(PROB_OMEGAS, PROB_CUMULATIVE):
        if u < c:
            return om
    return PROB_OMEGAS[-1]


ENUM_OMEGAS = tuple(0.5 * i for i in range(19))  # {0, 0.5, ..., 9}, Sec. 5.2.2


# --------------------------------------------------------------------------
# Algorithm 2 (Algorithm 1 is omega = 0)
# --------------------------------------------------------------------------

def _centred(X):
    return X - X.mean(axis=0, keepdims=True)


def criterion(stop: int, X_old, X_new, f_old: float, f_new: float) -> float:
    """Termination criterion after one iteration.

    STOP_REL_DISP:   ||c(X_new) - c(X_old)||_F / ||c(X_new)||_F, c = centring.
    STOP_REL_STRESS: (f_old - f_new) / f_old.
    A zero denominator gives 0 (nothing left to move or reduce).
    """
    if stop == STOP_REL_DISP:
        a, b = _centred(X_new), _centred(X_old)
        den = float(np.sqrt(np.sum(a * a)))
        return 0.0 if den == 0.0 else float(np.sqrt(np.sum((a - b) ** 2))) / den
    if stop == STOP_REL_STRESS:
        return 0.0 if f_old == 0.0 else (f_old - f_new) / f_old
    raise ValueError("unknown stop rule")


@dataclass
class RunResult:
    X: np.ndarray
    iterations: int
    stress: float
    trace_f: list = field(default_factory=list)       # f(X^0), f(X^1), ...
    trace_accept: list = field(default_factory=list)  # line 6 outcome per iteration
    trace_omega: list = field(default_factory=list)   # omega used per iteration
    trace_crit: list = field(default_factory=list)    # termination criterion per iteration
    trace_fH: list = field(default_factory=list)      # f(H(X^k)) per iteration
    converged: bool = False


def extrapolate(Z, X, omega: float, m=None) -> np.ndarray:
    """Line 5 of Algorithm 2.  Without m: Eq. (10), (1 + omega) Z - omega X.
    With per-vertex factors m (Sec. 6, first item of further work): vertex i
    moves by its own stride, x~_i = z_i + omega_i (z_i - x_i), with
    omega_i = omega * m_i."""
    Z, X = _f64(Z), _f64(X)
    if m is None:
        return (1.0 + omega) * Z - omega * X
    om_i = omega * np.asarray(m, dtype=np.float64).reshape(-1, 1)
    return Z + om_i * (Z - X)


def sor_step(X, D, omega_k: float, strategy: int = OMEGA_FIXED, solver=None, omega_vertex=None):
    """One pass of Algorithm 2's loop body: lines 4-8.  omega_vertex: None,
    or the per-vertex factors m of `extrapolate`.

    Returns (X_next, f(X_next), accepted, omega_used, f(H(X))).
    """
    X = _f64(X)
    solver = solver or PinnedSolver(D)
    Z = solver.solve(rhs(X, D))                      # line 4, Eq. (2-5)
    fZ = stress(Z, D)
    if strategy == OMEGA_ENUM:                        # Sec. 5.2.2
        best_f, best_om, best_X = None, None, None
        for om in ENUM_OMEGAS:
            Xt = extrapolate(Z, X, om, omega_vertex)
            ft = stress(Xt, D)
            if best_f is None or ft < best_f:
                best_f, best_om, best_X = ft, om, Xt
        return best_X, best_f, best_om > 0.0, best_om, fZ
    Xt = extrapolate(Z, X, omega_k, omega_vertex)     # line 5, Eq. (10)
    ft = stress(Xt, D)
    if ft <= fZ:                                      # line 6
        return Xt, ft, True, omega_k, fZ              # line 7
    return Z, fZ, False, omega_k, fZ


def sor_run(D, X0, omega: float = 0.0, strategy: int = OMEGA_FIXED, seed: int = 0,
            stop: int = STOP_REL_DISP, tol: float = 1e-4, max_iter: int = 1000,
            solver: PinnedSolver | None = None, omega_vertex=None) -> RunResult:
    """Algorithm 2 from X^0 until the criterion drops below tol or max_iter
    iterations ran.  omega = 0 with the fixed strategy is Algorithm 1.
    omega_vertex: per-vertex factors m (omega_i = omega m_i, Sec. 6)."""
    D = _f64(D)
    X = _f64(X0).copy()
    solver = solver or PinnedSolver(D)
    f = stress(X, D)
    res = RunResult(X=X, iterations=0, stress=f, trace_f=[f])
    for k in range(max_iter):
        om = omega_draw(seed, k) if strategy == OMEGA_PROB else omega
        Xn, fn, acc, om_used, fZ = sor_step(X, D, om, strategy, solver, omega_vertex)
        crit = criterion(stop, X, Xn, f, fn)
        res.trace_f.append(fn)
        res.trace_accept.append(bool(acc))
        res.trace_omega.append(float(om_used))
        res.trace_crit.append(float(crit))
        res.trace_fH.append(float(fZ))
        X, f = Xn, fn
        res.iterations = k + 1
        if crit < tol:
            res.converged = True
            break
    res.X, res.stress = X, f
    return res


# --------------------------------------------------------------------------
# Derivative of the stress with respect to edge lengths
# --------------------------------------------------------------------------

def _shortest_path_trees(rp, ci, ln):
    """For every source: Dijkstra distances and predecessors (the lowest-index
    tight neighbour).  Connected graphs only."""
    import heapq

    n = rp.shape[0] - 1
    out = []
    for s in range(n):
        dist = np.full(n, np.inf)
        dist[s] = 0.0
        heap = [(0.0, s)]
        done = np.zeros(n, dtype=bool)
        while heap:
            du, u = heapq.heappop(heap)
            if done[u]:
                continue
            done[u] = True
            for e in range(rp[u], rp[u + 1]):
                v = int(ci[e])
                c = du + ln[e]
                if c < dist[v]:
                    dist[v] = c
                    heapq.heappush(heap, (c, v))
        if not np.all(np.isfinite(dist)):
            raise ValueError("a connected graph is needed")
        pred = np.full(n, -1, dtype=np.int64)
        for v in range(n):
            if v == s:
                continue
            best = None
            for e in range(rp[v], rp[v + 1]):
                u = int(ci[e])
                if u != v and dist[u] + ln[e] == dist[v] and (best is None or u < best):
                    best = u
            if best is None:  # rounding: take the neighbour closest to tight
                best = min((abs(dist[int(ci[e])] + ln[e] - dist[v]), int(ci[e])) for e in range(rp[v], rp[v + 1]))[1]
            pred[v] = best
        out.append((dist, pred))
    return out


def pair_to_edge_grad(row_ptr, col_idx, edge_len, G) -> np.ndarray:
    """d L / d l_e from pair sensitivities G[i, j] = d L / d d_ij (symmetric
    n x n) when d_ij is the weighted shortest-path length (Sec. 5.4): every
    pair's path is walked back edge by edge (ties between paths have measure
    zero; the lower predecessor index is taken).  One value per CSR entry,
    equal for the two entries of an edge.  Connected graphs, small n."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    ln = _f64(edge_len)
    n = rp.shape[0] - 1
    entry = {}
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(ci[e])
            if v != u:
                entry.setdefault((min(u, v), max(u, v)), []).append(e)
    g_edge = {k: 0.0 for k in entry}
    for s, (dist, pred) in enumerate(_shortest_path_trees(rp, ci, ln)):
        for t in range(n):
            if t == s:
                continue
            v = t
            while v != s:
                u = int(pred[v])
                g_edge[(min(u, v), max(u, v))] += 0.5 * G[s, t]  # every pair is met from both ends
                v = u
    out = np.zeros(len(ci), dtype=np.float64)
    for k, es in entry.items():
        for e in es:
            out[e] = g_edge[k]
    return out


def stress_length_grad(X, row_ptr, col_idx, edge_len) -> np.ndarray:
    """d f / d l_e for Eq. (1) when d_ij is the weighted shortest-path length
    (Sec. 5.4) and w_ij = d_ij^-2 (Sec. 5.1).

    f = sum_{i<j} (r_ij / d_ij - 1)^2, so d f / d d_ij = -2 r_ij (r_ij - d_ij) / d_ij^3,
    and d d_ij / d l_e = 1 when e lies on the shortest path of (i, j) (0
    otherwise).  Returns one value per CSR entry, equal for the two entries
    of an undirected edge.  Connected graphs, small n.
    """
    X = _f64(X)
    _, D = apsp(row_ptr, col_idx, edge_len=edge_len)
    n = X.shape[0]
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                r = float(np.linalg.norm(X[i] - X[j]))
                G[i, j] = -2.0 * r * (r - D[i, j]) / D[i, j] ** 3
    return pair_to_edge_grad(row_ptr, col_idx, edge_len, G)


# --------------------------------------------------------------------------
# Unrolled differentiation of Algorithm 2 (the acceptance of line 6 held fixed)
# --------------------------------------------------------------------------

def unrolled_run(D, X0, K: int, omega: float, omega_vertex=None):
    """K iterations of Algorithm 2 with exact solves; returns the layouts
    X^0..X^K, the H-step outputs Z^1..Z^K and the acceptance of each step.
    omega_vertex: per-vertex factors m (omega_i = omega m_i, Sec. 6)."""
    solver = PinnedSolver(D)
    Xs, Zs, acc = [_f64(X0).copy()], [], []
    for _ in range(K):
        X = Xs[-1]
        Xn, fn, a, om, fZ = sor_step(X, D, omega, OMEGA_FIXED, solver, omega_vertex)
        Z = solver.solve(rhs(X, D))
        Xs.append(Xn)
        Zs.append(Z)
        acc.append(bool(a))
    return Xs, Zs, acc


def unrolled_adjoint(D, Xs, Zs, acc, omega: float, Xbar_K, omega_vertex=None):
    """Backward pass of unrolled_run: returns dL/dX^0 and the pair
    sensitivities dL/dd_ij (symmetric n x n) summed over the steps.

    Per step (Eq. (2-5), pinning, Eq. (10)): Zb = (1+omega) Xb' or Xb', Xb = -omega Xb'
    or 0 (omega_i = omega m_i per vertex with factors m); Yb = Zb - e_0 (1^T Zb);
    L^W lam = Yb; Xb += J_b(X)^T lam with b_i = sum_j (1/d_ij) (x_i - x_j)/r_ij;
    dL/dd_ij += -(dlam . u)/d^2 + 2 (dlam . dY)/d^3.  Plain loops over pairs."""
    D = _f64(D)
    n = D.shape[0]
    solver = PinnedSolver(D)
    Xb1 = _f64(Xbar_K).copy()
    Gd = np.zeros((n, n))
    om = omega if omega_vertex is None else omega * np.asarray(omega_vertex, dtype=np.float64).reshape(-1, 1)
    for k in reversed(range(len(acc))):
        X, Y = Xs[k], Zs[k]
        if acc[k]:
            Zb, Xb = (1.0 + om) * Xb1, -om * Xb1
        else:
            Zb, Xb = Xb1.copy(), np.zeros_like(Xb1)
        Yb = Zb.copy()
        Yb[0] -= Zb.sum(axis=0)
        lam = solver.solve(Yb)
        for i in range(n):
            for j in range(i + 1, n):
                d = D[i, j]
                dx = X[i] - X[j]
                dl = lam[i] - lam[j]
                g = 2.0 * float(dl @ (Y[i] - Y[j])) / d ** 3
                r = float(np.linalg.norm(dx))
                if r > 0.0:
                    u = dx / r
                    ul = float(u @ dl)
                    g -= ul / d ** 2
                    v = (dl - u * ul) / (d * r)
                    Xb[i] += v
                    Xb[j] -= v
                Gd[i, j] += g
                Gd[j, i] += g
        Xb1 = Xb
    return Xb1, Gd
