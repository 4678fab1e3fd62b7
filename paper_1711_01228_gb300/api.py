"""Python binding of the C ABI in include/fd_layout.h (argument marshalling only).

Every computation runs in ``libfdlayout.so`` (CUDA kernels for sm_103a); this
module only converts arrays to pointers and status codes to exceptions.  There
is no CPU fallback: if the library is missing, :func:`lib` raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
positions are float32 ``[n, dim]``, graphs int32 CSR.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

FD_OK = 0
STATUS_NAMES = {
    0: "FD_OK", 1: "FD_ERR_ARG", 2: "FD_ERR_CSR", 3: "FD_ERR_DISCONNECTED", 4: "FD_ERR_NONFINITE",
    5: "FD_ERR_CG_BREAKDOWN", 6: "FD_ERR_CG_MAXITER", 7: "FD_ERR_TIMEOUT", 8: "FD_ERR_OOM",
    9: "FD_ERR_CUDA", 10: "FD_ERR_UNIMPLEMENTED",
}
OMEGA_FIXED, OMEGA_PROB, OMEGA_ENUM = 0, 1, 2
STOP_REL_DISP, STOP_REL_STRESS = 0, 1
SOLVER_CG, SOLVER_DIRECT = 0, 1
DIRECT_MAX_N = 32768


class FdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


class Options(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("strategy", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("cg_max", ctypes.c_int32), ("cg_tol", ctypes.c_double), ("solver", ctypes.c_int32),
                ("first_iter", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("cg_steps", ctypes.c_int32), ("cg_maxed", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("pair_passes", ctypes.c_double), ("pairs", ctypes.c_double),
                ("final_stress", ctypes.c_double), ("final_crit", ctypes.c_double),
                ("matvec_passes", ctypes.c_double), ("stress_passes", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("cg_stalled", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("enum_candidate_passes", ctypes.c_double), ("rhs_skipped", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("dim", ctypes.c_int32), ("diameter", ctypes.c_int32),
                ("code_bytes", ctypes.c_int32), ("tile", ctypes.c_int32), ("num_tiles", ctypes.c_int32),
                ("distance_bytes", ctypes.c_int64), ("disconnected", ctypes.c_int32),
                ("sm_count", ctypes.c_int32), ("grid", ctypes.c_int32), ("tasks", ctypes.c_int32),
                ("apsp_ms", ctypes.c_double), ("stages", ctypes.c_int32), ("bfs_sweeps", ctypes.c_int32),
                ("factored", ctypes.c_int32), ("factor_ms", ctypes.c_double), ("tiles_per_stage", ctypes.c_int32),
                ("bfs_sources", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("num_graphs", ctypes.c_int32), ("dim", ctypes.c_int32), ("total_vertices", ctypes.c_int64),
                ("num_tiles", ctypes.c_int64), ("distance_bytes", ctypes.c_int64), ("max_n", ctypes.c_int32),
                ("max_diameter", ctypes.c_int32), ("disconnected", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("groups", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("graph_captured", ctypes.c_int32), ("apsp_ms", ctypes.c_double),
                ("small_tile_bytes", ctypes.c_int64), ("graphs_t128", ctypes.c_int32), ("graphs_t64", ctypes.c_int32),
                ("graphs_t32", ctypes.c_int32)]


EXPORTED = ["fd_options_default", "fd_layout_create", "fd_layout_destroy", "fd_energy", "fd_forces",
            "fd_sor_step", "fd_run", "fd_run_trace", "fd_distance_rows", "fd_layout_info",
            "fd_last_stats", "fd_last_error", "fd_status_string", "fd_energy_noalloc", "fd_timeline_enable",
            "fd_timeline_read", "fd_batch_create", "fd_batch_destroy", "fd_batch_run", "fd_batch_results",
            "fd_batch_tune", "fd_batch_set_shape", "fd_batch_distances", "fd_batch_get_info",
            "fd_batch_last_stats", "fd_energy_length_grad", "fd_sor_step_adjoint", "fd_adjoint_reset",
            "fd_adjoint_length_grad", "fd_set_vertex_omega", "fd_factor", "fd_factor_rows", "fd_factor_release",
            "fd_fp32_peak", "fd_run_trace_ext", "fd_batch_set_tiles", "fd_batch_get_tiles", "fd_batch_cached_tiles",
            "fd_batch_clear_tile_cache"]
GRAD_MAX_N = 131072
BATCH_MAX_N = 2048
BATCH_BUCKETS = 7          # size buckets of the tile-edge choice: n <= 32, 64, ..., 2048
BATCH_TILES = (32, 64, 128)
TIMELINE_TAGS = {1: "pack", 2: "stress", 3: "forces", 4: "rhs0", 5: "h_init", 6: "cg_au0", 7: "cg_step",
                 8: "candidates", 9: "vertex_phase"}
NOALLOC_MAX_N = 524288

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libfdlayout.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1711_01228_gb300.build.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(path)
    P, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    L.fd_options_default.argtypes = [ctypes.POINTER(Options)]
    L.fd_options_default.restype = None
    L.fd_layout_create.argtypes = [ctypes.POINTER(P), i32, i32, P, P, P, i32, P]
    L.fd_layout_create.restype = i32
    L.fd_layout_destroy.argtypes = [P]
    L.fd_layout_destroy.restype = None
    L.fd_energy.argtypes = [P, P, ctypes.POINTER(f64)]
    L.fd_energy.restype = i32
    L.fd_forces.argtypes = [P, P, P]
    L.fd_forces.restype = i32
    L.fd_sor_step.argtypes = [P, P, ctypes.POINTER(Options), i32, ctypes.POINTER(f64), ctypes.POINTER(i32),
                              ctypes.POINTER(f64)]
    L.fd_sor_step.restype = i32
    L.fd_run.argtypes = [P, P, ctypes.POINTER(Options), ctypes.POINTER(i32), ctypes.POINTER(f64), P]
    L.fd_run.restype = i32
    L.fd_set_vertex_omega.argtypes = [P, P]
    L.fd_set_vertex_omega.restype = i32
    L.fd_fp32_peak.argtypes = [i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.fd_fp32_peak.restype = i32
    L.fd_factor.argtypes = [P]
    L.fd_factor.restype = i32
    L.fd_factor_rows.argtypes = [P, i32, i32, P]
    L.fd_factor_rows.restype = i32
    L.fd_factor_release.argtypes = [P]
    L.fd_factor_release.restype = i32
    L.fd_run_trace.argtypes = [P, P, P, P, P]
    L.fd_run_trace.restype = i32
    L.fd_run_trace_ext.argtypes = [P, P, P, P]
    L.fd_run_trace_ext.restype = i32
    L.fd_distance_rows.argtypes = [P, i32, i32, P]
    L.fd_distance_rows.restype = i32
    L.fd_layout_info.argtypes = [P, ctypes.POINTER(Info)]
    L.fd_layout_info.restype = i32
    L.fd_last_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.fd_last_stats.restype = i32
    L.fd_last_error.argtypes = [P]
    L.fd_last_error.restype = i32
    L.fd_status_string.argtypes = [i32]
    L.fd_status_string.restype = ctypes.c_char_p
    L.fd_energy_noalloc.argtypes = [P, P, i32, i32, P, P]
    L.fd_energy_noalloc.restype = i32
    L.fd_timeline_enable.argtypes = [P, i32]
    L.fd_timeline_enable.restype = i32
    L.fd_timeline_read.argtypes = [P, P, i32, ctypes.POINTER(i32)]
    L.fd_timeline_read.restype = i32
    L.fd_batch_create.argtypes = [ctypes.POINTER(P), i32, i32, P, P, P, i32, P]
    L.fd_batch_create.restype = i32
    L.fd_batch_destroy.argtypes = [P]
    L.fd_batch_destroy.restype = None
    L.fd_batch_run.argtypes = [P, P, ctypes.POINTER(Options), P, P, P]
    L.fd_batch_run.restype = i32
    L.fd_batch_results.argtypes = [P, P, P, P, P, P, P, P]
    L.fd_batch_results.restype = i32
    L.fd_batch_tune.argtypes = [P, P, ctypes.POINTER(Options), i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.fd_batch_tune.restype = i32
    L.fd_batch_set_shape.argtypes = [P, i32, i32]
    L.fd_batch_set_shape.restype = i32
    L.fd_batch_set_tiles.argtypes = [P, P]
    L.fd_batch_set_tiles.restype = i32
    L.fd_batch_get_tiles.argtypes = [P, P]
    L.fd_batch_get_tiles.restype = i32
    L.fd_batch_cached_tiles.argtypes = [i32, P]
    L.fd_batch_cached_tiles.restype = i32
    L.fd_batch_clear_tile_cache.argtypes = []
    L.fd_batch_clear_tile_cache.restype = None
    L.fd_batch_distances.argtypes = [P, i32, P]
    L.fd_batch_distances.restype = i32
    L.fd_batch_get_info.argtypes = [P, ctypes.POINTER(BatchInfo)]
    L.fd_batch_get_info.restype = i32
    L.fd_batch_last_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.fd_batch_last_stats.restype = i32
    L.fd_energy_length_grad.argtypes = [P, P, P, ctypes.POINTER(f64)]
    L.fd_energy_length_grad.restype = i32
    L.fd_sor_step_adjoint.argtypes = [P, P, P, i32, f64, P, P, ctypes.POINTER(Options), ctypes.POINTER(i32)]
    L.fd_sor_step_adjoint.restype = i32
    L.fd_adjoint_reset.argtypes = [P]
    L.fd_adjoint_reset.restype = i32
    L.fd_adjoint_length_grad.argtypes = [P, P]
    L.fd_adjoint_length_grad.restype = i32
    _LIB = L
    return L


def torch_empty_like(a):
    """An uninitialised array of a's kind, shape and dtype."""
    if _is_torch(a):
        import torch
        return torch.empty_like(a)
    return np.empty_like(a)


def _check(status: int, where: str):
    if status != FD_OK:
        raise FdError(status, where)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype) -> int:
    """Pointer of a contiguous numpy array or torch tensor of the given dtype."""
    if a is None:
        return None
    if _is_torch(a):
        import torch
        want = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy {np.dtype(dtype).name} array")
    return a.ctypes.data


def options(**kw) -> Options:
    o = Options()
    lib().fd_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class RunResult:
    iterations: int
    stress: float
    trace_f: np.ndarray = field(default=None)
    accepted: np.ndarray = field(default=None)
    omega: np.ndarray = field(default=None)
    cg_steps: np.ndarray = field(default=None)
    crit: np.ndarray = field(default=None)
    f_h: np.ndarray = field(default=None)             # f(H(X^k)) per iteration
    f_extrapolated: np.ndarray = field(default=None)  # f of line 5's candidate per iteration
    t_ms: np.ndarray = field(default=None)            # device ms from the launch to the end of iteration k
    stats: dict = field(default_factory=dict)


class Layout:
    """A graph prepared for layout: ideal distances on the GPU plus scratch.

    ``row_ptr``/``col_idx`` int32 CSR (numpy, or torch host/CUDA tensors),
    ``edge_len`` optional float32 lengths, ``dim`` in {1, 2, 3}.
    """

    def __init__(self, row_ptr, col_idx, dim: int = 2, edge_len=None, disconnected_policy: int = 0,
                 stream=None):
        L = lib()
        n = int(row_ptr.shape[0]) - 1
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        status = L.fd_layout_create(ctypes.byref(h), n, int(dim), _ptr(row_ptr, np.int32),
                                    _ptr(col_idx, np.int32) if col_idx is not None and len(col_idx) else None,
                                    _ptr(edge_len, np.float32), int(disconnected_policy), st)
        _check(status, "fd_layout_create")
        self._h = h
        self.n, self.dim = n, int(dim)
        self._nnz = int(row_ptr[-1])

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().fd_layout_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- queries
    def info(self) -> dict:
        i = Info()
        _check(lib().fd_layout_info(self._h, ctypes.byref(i)), "fd_layout_info")
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def stats(self) -> dict:
        s = Stats()
        _check(lib().fd_last_stats(self._h, ctypes.byref(s)), "fd_last_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def timeline_enable(self, cap: int = 100000):
        """Record (phase tag, ns) at every grid barrier of later launches."""
        _check(lib().fd_timeline_enable(self._h, int(cap)), "fd_timeline_enable")
        self._tl_cap = int(cap)

    def timeline(self) -> np.ndarray:
        """[k, 2] array of (tag, ns since launch start) of the last launch."""
        cap = getattr(self, "_tl_cap", 0)
        out = np.zeros((max(cap, 1), 2), dtype=np.float64)
        k = ctypes.c_int32()
        _check(lib().fd_timeline_read(self._h, out.ctypes.data, cap, ctypes.byref(k)), "fd_timeline_read")
        return out[: min(k.value, cap)]

    def distance_rows(self, row0: int, nrows: int) -> np.ndarray:
        out = np.empty((nrows, self.n), dtype=np.float64)
        _check(lib().fd_distance_rows(self._h, int(row0), int(nrows), out.ctypes.data), "fd_distance_rows")
        return out

    # -- the method
    def _xcheck(self, X):
        if tuple(X.shape) != (self.n, self.dim):
            raise ValueError(f"X must have shape ({self.n}, {self.dim})")

    def energy(self, X) -> float:
        """Stress f(X), Eq. (1)."""
        self._xcheck(X)
        f = ctypes.c_double()
        _check(lib().fd_energy(self._h, _ptr(X, np.float32), ctypes.byref(f)), "fd_energy")
        return f.value

    def forces(self, X, out=None):
        """F = (L^X - L^W) X; returns an array of X's kind unless ``out`` is given."""
        self._xcheck(X)
        if out is None:
            if _is_torch(X):
                import torch
                out = torch.empty_like(X)
            else:
                out = np.empty_like(X)
        _check(lib().fd_forces(self._h, _ptr(X, np.float32), _ptr(out, np.float32)), "fd_forces")
        return out

    def length_grad(self, X, out=None):
        """d f / d l_e for every CSR entry of a weighted graph (equal for the
        two entries of an edge); returns (f, grad) with grad of X's kind
        unless ``out`` is given."""
        self._xcheck(X)
        if out is None:
            nnz = self._nnz
            if _is_torch(X):
                import torch
                out = torch.empty(nnz, dtype=torch.float32, device=X.device)
            else:
                out = np.empty(nnz, dtype=np.float32)
        f = ctypes.c_double()
        _check(lib().fd_energy_length_grad(self._h, _ptr(X, np.float32), _ptr(out, np.float32), ctypes.byref(f)),
               "fd_energy_length_grad")
        return f.value, out

    def sor_step_adjoint(self, X_k, X_k1, accepted: bool, omega: float, Xbar_k1, out=None, **opts):
        """dL/dX_k from dL/dX_k1 through one iteration of Algorithm 2 (acceptance
        held fixed); adds the pair sensitivities to the accumulator after
        adjoint_reset().  Returns (Xbar_k, CG steps of the adjoint solve)."""
        if out is None:
            out = torch_empty_like(X_k)
        o = options(**opts)
        cg = ctypes.c_int32()
        _check(lib().fd_sor_step_adjoint(self._h, _ptr(X_k, np.float32), _ptr(X_k1, np.float32), int(bool(accepted)),
                                         float(omega), _ptr(Xbar_k1, np.float32), _ptr(out, np.float32),
                                         ctypes.byref(o), ctypes.byref(cg)), "fd_sor_step_adjoint")
        return out, cg.value

    def adjoint_reset(self):
        _check(lib().fd_adjoint_reset(self._h), "fd_adjoint_reset")

    def adjoint_length_grad(self, out=None):
        """dL/dl_e from the pair sensitivities accumulated since adjoint_reset()."""
        if out is None:
            out = np.empty(self._nnz, dtype=np.float32)
        _check(lib().fd_adjoint_length_grad(self._h, _ptr(out, np.float32)), "fd_adjoint_length_grad")
        return out

    def factor(self) -> float:
        """Inverts the shifted L^W once on the device for solver=SOLVER_DIRECT;
        returns the device time in ms."""
        _check(lib().fd_factor(self._h), "fd_factor")
        return self.info()["factor_ms"]

    def factor_rows(self, row0: int, nrows: int) -> np.ndarray:
        """Rows of the factored inverse (L^W + sigma/n 1 1^T)^-1, float64 [nrows, n]."""
        out = np.empty((nrows, self.n), dtype=np.float64)
        _check(lib().fd_factor_rows(self._h, int(row0), int(nrows), out.ctypes.data), "fd_factor_rows")
        return out

    def factor_release(self):
        _check(lib().fd_factor_release(self._h), "fd_factor_release")

    def set_vertex_omega(self, m=None):
        """Per-vertex relaxation factors (Sec. 6): later runs use omega_i =
        omega * m[i] (m: n non-negative floats, host or device); None
        restores a single omega."""
        if m is None:
            _check(lib().fd_set_vertex_omega(self._h, None), "fd_set_vertex_omega")
            return
        if _is_torch(m):
            if m.numel() != self.n:
                raise ValueError("m must have n entries")
        else:
            m = np.ascontiguousarray(m, dtype=np.float32)
            if m.shape != (self.n,):
                raise ValueError("m must have n entries")
        _check(lib().fd_set_vertex_omega(self._h, _ptr(m, np.float32)), "fd_set_vertex_omega")

    def sor_step(self, X, k: int = 0, **opts):
        """One iteration of Algorithm 2 in place on X; returns (f, accepted, crit)."""
        self._xcheck(X)
        o = options(**opts)
        f, acc, crit = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().fd_sor_step(self._h, _ptr(X, np.float32), ctypes.byref(o), int(k), ctypes.byref(f),
                                 ctypes.byref(acc), ctypes.byref(crit)), "fd_sor_step")
        return f.value, bool(acc.value), crit.value

    def run(self, X, trace: bool = False, **opts) -> RunResult:
        """Algorithm 2 to convergence in place on X."""
        self._xcheck(X)
        o = options(**opts)
        iters, f = ctypes.c_int32(), ctypes.c_double()
        tf = np.zeros(o.max_iter + 1, dtype=np.float64) if trace else None
        _check(lib().fd_run(self._h, _ptr(X, np.float32), ctypes.byref(o), ctypes.byref(iters), ctypes.byref(f),
                            tf.ctypes.data if trace else None), "fd_run")
        res = RunResult(iterations=iters.value, stress=f.value, stats=self.stats())
        if trace:
            k = iters.value
            res.trace_f = tf[:k + 1].copy()
            acc = np.zeros(max(k, 1), dtype=np.int32)
            om = np.zeros(max(k, 1), dtype=np.float64)
            cg = np.zeros(max(k, 1), dtype=np.int32)
            cr = np.zeros(max(k, 1), dtype=np.float64)
            _check(lib().fd_run_trace(self._h, acc.ctypes.data, om.ctypes.data, cg.ctypes.data, cr.ctypes.data),
                   "fd_run_trace")
            res.accepted, res.omega, res.cg_steps, res.crit = acc[:k], om[:k], cg[:k], cr[:k]
            fh = np.zeros(max(k, 1), dtype=np.float64)
            ft = np.zeros(max(k, 1), dtype=np.float64)
            tm = np.zeros(max(k, 1), dtype=np.float64)
            _check(lib().fd_run_trace_ext(self._h, fh.ctypes.data, ft.ctypes.data, tm.ctypes.data), "fd_run_trace_ext")
            res.f_h, res.f_extrapolated, res.t_ms = fh[:k], ft[:k], tm[:k]
        return res


def fp32_peak(packed: bool = True) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s
    (two-wide packed FMAs when ``packed``)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().fd_fp32_peak(int(bool(packed)), ctypes.byref(t), ctypes.byref(ms)), "fd_fp32_peak")
    return t.value


def trace_records(result: RunResult) -> list:
    """Per-iteration records of a run made with ``trace=True``: iteration k
    (1-based), stress after it, f(H(X^k)) and f of the extrapolated
    candidate, whether line 6 kept the extrapolation, the omega used, CG
    steps of its H step, the termination criterion and the device time since
    the launch began."""
    if result.trace_f is None:
        raise ValueError("the run was made without trace=True")
    out = []
    for k in range(result.iterations):
        out.append({"k": k + 1, "stress": float(result.trace_f[k + 1]), "stress_h": float(result.f_h[k]),
                    "stress_extrapolated": float(result.f_extrapolated[k]), "accepted": bool(result.accepted[k]),
                    "omega": float(result.omega[k]), "cg_steps": int(result.cg_steps[k]),
                    "crit": float(result.crit[k]), "t_ms": float(result.t_ms[k])})
    return out


def write_trace_jsonl(result: RunResult, path: str, **extra) -> None:
    """One JSON line per iteration (``trace_records``), each with ``extra`` fields added."""
    import json

    with open(path, "w") as f:
        for rec in trace_records(result):
            rec.update(extra)
            f.write(json.dumps(rec) + "\n")


def energy_noalloc(X, D, stream=None) -> float:
    """Stress f(X) from a dense device distance matrix without any device
    allocation by the library (for callers whose GPU memory is owned by
    another allocator).  X: float32 CUDA tensor [n, dim]; D: float32 CUDA
    tensor [n, n] whose strictly lower triangle holds d_ij."""
    n, dim = int(X.shape[0]), int(X.shape[1])
    if tuple(D.shape) != (n, n):
        raise ValueError("D must be [n, n]")
    f = ctypes.c_double()
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().fd_energy_noalloc(_ptr(X, np.float32), _ptr(D, np.float32), n, dim, ctypes.addressof(f), st),
           "fd_energy_noalloc")
    return f.value


@dataclass
class BatchResult:
    iterations: np.ndarray      # [G] iterations per graph
    stress: np.ndarray          # [G] final stress per graph
    status: np.ndarray          # [G] fd_status per graph
    cg_steps: np.ndarray
    accepted: np.ndarray
    crit: np.ndarray
    matvec_passes: np.ndarray
    stress_passes: np.ndarray
    graph_ms: np.ndarray        # [G] device time spent on each graph
    stats: dict = field(default_factory=dict)


class Batch:
    """Many independent graphs (each at most BATCH_MAX_N vertices) laid out in
    one persistent launch.

    ``graph_ptr`` int32 [G+1] vertex offsets; ``row_ptr``/``col_idx`` the
    concatenated int32 CSR with global vertex ids (edges stay inside graphs).
    """

    def __init__(self, graph_ptr, row_ptr, col_idx, dim: int = 2, disconnected_policy: int = 0, stream=None):
        L = lib()
        G = int(graph_ptr.shape[0]) - 1
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        status = L.fd_batch_create(ctypes.byref(h), G, int(dim), _ptr(graph_ptr, np.int32), _ptr(row_ptr, np.int32),
                                   _ptr(col_idx, np.int32) if col_idx is not None and len(col_idx) else None,
                                   int(disconnected_policy), st)
        _check(status, "fd_batch_create")
        self._h = h
        self.G, self.dim = G, int(dim)
        gp = graph_ptr.cpu().numpy() if _is_torch(graph_ptr) else np.asarray(graph_ptr)
        self.sizes = np.diff(gp.astype(np.int64))
        self.graph_ptr = gp.astype(np.int64)
        self.N = int(gp[-1])

    @classmethod
    def from_graphs(cls, graphs, dim: int = 2, disconnected_policy: int = 0, stream=None):
        """Batch from a list of (row_ptr, col_idx) numpy CSR pairs."""
        gp, rp, ci = concat_graphs(graphs)
        return cls(gp, rp, ci, dim=dim, disconnected_policy=disconnected_policy, stream=stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().fd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        i = BatchInfo()
        _check(lib().fd_batch_get_info(self._h, ctypes.byref(i)), "fd_batch_get_info")
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def stats(self) -> dict:
        s = Stats()
        _check(lib().fd_batch_last_stats(self._h, ctypes.byref(s)), "fd_batch_last_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def distances(self, g: int) -> np.ndarray:
        """Stored hop distances of graph g, [n_g, n_g] float64."""
        n = int(self.sizes[g])
        out = np.empty((n, n), dtype=np.float64)
        _check(lib().fd_batch_distances(self._h, int(g), out.ctypes.data), "fd_batch_distances")
        return out

    def set_shape(self, groups: int, stages: int):
        _check(lib().fd_batch_set_shape(self._h, int(groups), int(stages)), "fd_batch_set_shape")

    def set_tiles(self, tiles):
        """Tile edge (32, 64 or 128) of each of the BATCH_BUCKETS size buckets."""
        t = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(BATCH_BUCKETS))
        _check(lib().fd_batch_set_tiles(self._h, t.ctypes.data), "fd_batch_set_tiles")

    def tiles(self) -> list:
        t = np.zeros(BATCH_BUCKETS, dtype=np.int32)
        _check(lib().fd_batch_get_tiles(self._h, t.ctypes.data), "fd_batch_get_tiles")
        return t.tolist()

    def tune(self, X, probe_iter: int = 5, repeats: int = 2, **opts):
        """The autotuner: times every feasible launch shape on X and keeps the
        fastest, then the tile edge of each size bucket (read back with
        tiles()); returns (groups, stages)."""
        o = options(**opts)
        g, s = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fd_batch_tune(self._h, _ptr(X, np.float32), ctypes.byref(o), int(probe_iter), int(repeats),
                                   ctypes.byref(g), ctypes.byref(s)), "fd_batch_tune")
        return g.value, s.value

    def run(self, X, omega=None, check: bool = True, **opts) -> BatchResult:
        """Algorithm 2 on every graph, in place on X ([N, dim] float32).
        ``omega``: None (the default option), one number for every graph, or a
        float64 array [G] of per-graph omegas."""
        if tuple(X.shape) != (self.N, self.dim):
            raise ValueError(f"X must have shape ({self.N}, {self.dim})")
        G = self.G
        om = None
        if omega is not None:
            if not _is_torch(omega) and np.ndim(omega) == 0:
                opts["omega"] = float(omega)  # one omega for every graph
            else:
                om = omega if _is_torch(omega) else np.ascontiguousarray(omega, dtype=np.float64)
                if tuple(om.shape) != (G,):
                    raise ValueError(f"per-graph omega must have shape ({G},)")
        o = options(**opts)
        it = np.zeros(G, dtype=np.int32)
        f = np.zeros(G, dtype=np.float64)
        status = lib().fd_batch_run(self._h, _ptr(X, np.float32), ctypes.byref(o),
                                    _ptr(om, np.float64) if om is not None else None, it.ctypes.data, f.ctypes.data)
        if check:
            _check(status, "fd_batch_run")
        st = np.zeros(G, dtype=np.int32)
        cg = np.zeros(G, dtype=np.int32)
        acc = np.zeros(G, dtype=np.int32)
        cr = np.zeros(G, dtype=np.float64)
        mv = np.zeros(G, dtype=np.float64)
        sp = np.zeros(G, dtype=np.float64)
        gm = np.zeros(G, dtype=np.float64)
        _check(lib().fd_batch_results(self._h, st.ctypes.data, cg.ctypes.data, acc.ctypes.data, cr.ctypes.data,
                                      mv.ctypes.data, sp.ctypes.data, gm.ctypes.data), "fd_batch_results")
        return BatchResult(iterations=it, stress=f, status=st, cg_steps=cg, accepted=acc, crit=cr,
                           matvec_passes=mv, stress_passes=sp, graph_ms=gm, stats=self.stats())


def concat_graphs(graphs):
    """(graph_ptr, row_ptr, col_idx) of the disjoint union of CSR graphs."""
    sizes = [len(rp) - 1 for rp, _ in graphs]
    gp = np.zeros(len(graphs) + 1, dtype=np.int32)
    gp[1:] = np.cumsum(sizes)
    rps, cis = [np.zeros(1, dtype=np.int64)], []
    e0 = 0
    for (rp, ci), v0 in zip(graphs, gp[:-1]):
        rps.append(np.asarray(rp[1:], dtype=np.int64) + e0)
        cis.append(np.asarray(ci, dtype=np.int64) + int(v0))
        e0 += int(rp[-1])
    rp_all = np.concatenate(rps).astype(np.int32)
    ci_all = np.concatenate(cis).astype(np.int32) if cis else np.zeros(0, dtype=np.int32)
    return gp, rp_all, ci_all


def batch_cached_tiles(dim: int) -> list:
    """Tile edges tuned in this process for layout dimension dim (0: not tuned)."""
    t = np.zeros(BATCH_BUCKETS, dtype=np.int32)
    _check(lib().fd_batch_cached_tiles(int(dim), t.ctypes.data), "fd_batch_cached_tiles")
    return t.tolist()


def batch_clear_tile_cache():
    lib().fd_batch_clear_tile_cache()
