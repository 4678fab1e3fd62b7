/*
 * fd_layout.h -- C ABI of the GB300 (sm_103a) stress-majorization layout
 * engine with successive over-relaxation.
 *
 * Method: Wang & Wang, "A Fast Successive Over-Relaxation Algorithm for
 * Force-Directed Network Graph Drawing", Sci. China Inf. Sci. 55:677 (2012).
 *
 *   stress   f(X) = sum_{i<j} w_ij (||x_i - x_j|| - d_ij)^2           Sec. 2, Eq. (1)
 *   weights  w_ij = d_ij^{-2}                                         Sec. 5.1
 *   d_ij     shortest-path length in the graph (hop count, or the sum
 *            of edge lengths when lengths are given)                  Sec. 2, Sec. 5.4
 *   step H   solve L^W X^{k+1} = L^{X^k} X^k, first vertex pinned      Prop. 2.3, Eq. (2-5)
 *   SOR      X~ = (1 + omega) X^{k+1} - omega X^k, kept iff
 *            f(X~) <= f(X^{k+1})                                       Algorithm 2, Eq. (10)
 *   per-vertex omega_i = omega m_i                                      Sec. 6
 *   solvers  CG, or the inverse of the shifted L^W made once          Sec. 2
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers may be host or device (CUDA) memory; the library detects which
 *    with cudaPointerGetAttributes and copies host data in and out on its
 *    stream.  Ownership never transfers: the library never frees a caller
 *    pointer and keeps none after the call returns.
 *  - Vertices are 0-based.  Positions are float32, row-major [n][dim],
 *    dim in {1, 2, 3}.
 *  - Graphs are int32 CSR: row_ptr[n+1] (row_ptr[0] = 0, non-decreasing),
 *    col_idx[row_ptr[n]] with 0 <= col_idx < n.  The graph must be
 *    undirected: every (u, v) entry needs a (v, u) entry (with the same
 *    length when lengths are given).  Self loops and repeated entries are
 *    allowed and ignored.
 *  - All GPU work runs on the CUDA stream given at creation (NULL = the
 *    legacy default stream) on the device that was current at creation.
 *    Every call returns only after its results are on the host (the stream
 *    is synchronised), so host scalars are valid on return.
 *  - Errors are returned as fd_status; the handle also keeps the last
 *    error.  The library never aborts the process and never traps on the
 *    GPU: device-side failures (non-finite values, a wait that timed out)
 *    come back as status codes.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef FD_LAYOUT_H
#define FD_LAYOUT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fd_layout fd_layout; /* opaque; owns the distance tiles and all scratch */

typedef enum {
  FD_OK = 0,
  FD_ERR_ARG = 1,           /* bad argument (null pointer, dim out of range, n < 1, ...) */
  FD_ERR_CSR = 2,           /* malformed or non-symmetric CSR, bad edge length */
  FD_ERR_DISCONNECTED = 3,  /* graph not connected and disconnected_policy == 0 */
  FD_ERR_NONFINITE = 4,     /* NaN/Inf in the positions or in a computed stress */
  FD_ERR_CG_BREAKDOWN = 5,  /* the linear solve broke down: p^T L^W p <= 0 in CG, or a pivot of fd_factor <= 0 */
  FD_ERR_CG_MAXITER = 6,    /* reserved (a solve that hits cg_max is counted, not fatal) */
  FD_ERR_TIMEOUT = 7,       /* a device-side grid barrier wait exceeded its time limit */
  FD_ERR_OOM = 8,           /* device or host allocation failed */
  FD_ERR_CUDA = 9,          /* other CUDA runtime error */
  FD_ERR_UNIMPLEMENTED = 10 /* option not supported by this build */
} fd_status;

/* How omega is chosen each iteration (Sec. 5.2). */
typedef enum {
  FD_OMEGA_FIXED = 0, /* omega constant over the run (Sec. 5.2.1); omega = 0 is Algorithm 1 */
  FD_OMEGA_PROB = 1,  /* roulette over P(0.5)=P(1)=0.3, P(1.5)=P(2)=0.2 (Sec. 5.2.3) */
  FD_OMEGA_ENUM = 2   /* argmin of f over omega in {0, 0.5, ..., 9} (Sec. 5.2.2), ties to the smaller omega;
                         X^{k+1} is the argmin ("accepted" when it is not omega = 0) */
} fd_omega_strategy;

/* Solver of Eq. (2-5) (Sec. 2 names Cholesky factorisation, CG and
 * Gauss-Seidel).  FD_SOLVER_DIRECT needs fd_factor on the handle first. */
typedef enum {
  FD_SOLVER_CG = 0,     /* Jacobi-preconditioned CG, warm-started from the previous layout */
  FD_SOLVER_DIRECT = 1  /* refinement with the inverse made by fd_factor: x += A'^-1 r, r -= L^W (A'^-1 r) */
} fd_solver;

/* Termination rule.  The paper leaves it open ("until some termination
 * conditions were satisfied", Algorithms 1 and 2); these are the library's
 * two readings, each tested after every iteration. */
typedef enum {
  FD_STOP_REL_DISP = 0,  /* ||c(X^{k+1}) - c(X^k)||_F / ||c(X^{k+1})||_F < tol, c = centring */
  FD_STOP_REL_STRESS = 1 /* (f(X^k) - f(X^{k+1})) / f(X^k) < tol */
} fd_stop_rule;

typedef struct {
  double omega;      /* the paper's omega >= 0 (Eq. (10)); classical SOR factor is 1 + omega */
  int32_t strategy;  /* fd_omega_strategy */
  int32_t stop;      /* fd_stop_rule */
  uint64_t seed;     /* FD_OMEGA_PROB: draw k uses SplitMix64(seed), k-th output */
  double tol;        /* termination threshold (see fd_stop_rule) */
  int32_t max_iter;  /* maximum outer iterations (each one H step) */
  int32_t cg_max;    /* maximum conjugate-gradient (or refinement) steps per H step */
  double cg_tol;     /* the H solve stops when ||r_c|| <= cg_tol * ||b_c|| for every column c */
  int32_t solver;    /* fd_solver: how Eq. (2-5) is solved in every H step */
  int32_t first_iter; /* fd_run: index k of its first iteration (FD_OMEGA_PROB draws the k-th
                         output), so that a run checkpointed after k iterations (its X) resumes
                         with the same omega sequence; 0 for a fresh run */
} fd_options;

/* Statistics of the last fd_run / fd_sor_step / fd_energy / fd_forces call. */
typedef struct {
  int32_t iterations;      /* outer iterations performed */
  int32_t cg_steps;        /* total CG steps over all H solves */
  int32_t cg_maxed;        /* H solves that stopped at cg_max before reaching cg_tol */
  int32_t accepted;        /* iterations whose extrapolation was kept (line 6 true) */
  double pair_passes;      /* all-pairs passes evaluated (matvec = 1, stress/RHS per candidate = 1,
                              enumeration: 1 per candidate stress) */
  double pairs;            /* unordered vertex pairs per pass: n (n - 1) / 2 */
  double final_stress;     /* f at the returned layout */
  double final_crit;       /* last termination criterion value */
  double matvec_passes;    /* passes of y = L^W p (inside the H solves) */
  double stress_passes;    /* passes of stress (+ L^X X or force) per candidate layout */
  double kernel_ms;        /* device time of the call's layout kernel (CUDA events on the handle's stream) */
  int32_t cg_stalled;      /* CG columns stopped before cg_tol because rounding left no descent */
  int32_t reserved;
  double enum_candidate_passes; /* FD_OMEGA_ENUM: candidate stresses evaluated by the enumeration passes
                              (19 per pass, stress only; not in stress_passes) */
  double rhs_skipped;      /* candidate evaluations counted in stress_passes whose right-hand side was
                              not computed: the two-candidate pass computes only the extrapolated
                              layout's (one per such pass) */
} fd_stats;

/* Library facts about a handle. */
typedef struct {
  int32_t n, dim;
  int32_t diameter;        /* largest finite d_ij (hop count; rounded up when weighted) */
  int32_t code_bytes;      /* bytes per stored pair: 1 (uint8 hop counts) or 4 (float32) */
  int32_t tile;            /* vertices per tile side */
  int32_t num_tiles;       /* stored tiles (unordered tile pairs) */
  int64_t distance_bytes;  /* device bytes of the stored distance tiles */
  int32_t disconnected;    /* 1 if some pairs were unreachable and filled by policy 1 */
  int32_t sm_count;        /* SMs of the device */
  int32_t grid;            /* CTAs of the cooperative layout kernel */
  int32_t tasks;           /* work items (runs of tiles) per all-pairs pass */
  double apsp_ms;          /* device time of the shortest-path kernel at creation (CUDA events) */
  int32_t stages;          /* tiles in flight per CTA in the layout kernel's copy pipeline (2 to 4) */
  int32_t bfs_sweeps;      /* unit edges: passes over the edge list summed over the multi-source searches */
  int32_t factored;        /* 1 after fd_factor (FD_SOLVER_DIRECT available) */
  double factor_ms;        /* device time of the last fd_factor (CUDA events) */
  int32_t tiles_per_stage; /* consecutive tiles of a task per pipeline stage (1 or 2) */
  int32_t bfs_sources;     /* unit edges: sources per multi-source search: 64 (one search per CTA) or
                              256 (one search over all CTAs, a grid barrier per level; n >= 65536 and
                              vertex 0's eccentricity <= 32) */
} fd_info;

/* Fills *opt with the defaults: omega 0.5, FIXED, REL_DISP, seed 0,
 * tol 1e-4, max_iter 1000, cg_max 200, cg_tol 1e-6, FD_SOLVER_CG, first_iter 0. */
void fd_options_default(fd_options* opt);

/* Builds a handle for graph G = (V, E) with n vertices laid out in dim
 * dimensions: validates the CSR, computes every ideal distance d_ij as a
 * shortest-path length (multi-source BFS on the GPU; label-correcting
 * relaxation when edge_len is given) and the row sums s_i = sum_j w_ij of
 * L^W (Prop. 2.1).  Sec. 2, Eq. (1); w = d^-2 per Sec. 5.1.
 *   out        receives the handle (NULL on failure)
 *   n          number of vertices (>= 1)
 *   dim        layout dimension, 1..3
 *   row_ptr    int32[n+1], host or device
 *   col_idx    int32[row_ptr[n]], host or device
 *   edge_len   float32[row_ptr[n]] positive finite lengths, or NULL for unit edges
 *   disconnected_policy  0: FD_ERR_DISCONNECTED if some pair is unreachable;
 *                        1: unreachable pairs get d = (largest finite d) + 1
 *   cuda_stream cudaStream_t to run on, or NULL
 * Errors: FD_ERR_ARG, FD_ERR_CSR, FD_ERR_DISCONNECTED, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_layout_create(fd_layout** out, int32_t n, int32_t dim, const int32_t* row_ptr,
                           const int32_t* col_idx, const float* edge_len,
                           int32_t disconnected_policy, void* cuda_stream);

/* Releases every device and host resource of the handle (NULL is a no-op). */
void fd_layout_destroy(fd_layout* h);

/* Stress f(X) of Eq. (1) at X (float32 [n][dim], host or device), written
 * to *f_out (host).  Errors: FD_ERR_ARG, FD_ERR_NONFINITE, FD_ERR_CUDA. */
fd_status fd_energy(fd_layout* h, const float* X, double* f_out);

/* Largest n accepted by fd_energy_noalloc (its scratch holds one partial sum
 * per 128 vertices: 4096 doubles plus one, 32 KB per device). */
#define FD_NOALLOC_MAX_N 524288

/* Stress f(X) like fd_energy, for callers that cannot allocate GPU memory.
 * The paper has no counterpart to this entry point; it is a library
 * convenience.  Some callers cannot call cudaMalloc: code inside a process
 * whose device memory is owned by another allocator (a framework's caching
 * allocator, a fixed-size arena), where one more allocation may fail or
 * synchronise the whole device, and latency-critical loops that cannot
 * afford one.  This call allocates nothing and needs no handle: its only
 * scratch is a fixed 32 KB array in the library's device image, which every
 * GPU that loads the library keeps until the process exits.
 *   X       float32 [n][dim], memory of the current device (or managed)
 *   D       float32 [n][n], memory of the current device (or managed),
 *           row-major; only the strictly lower triangle is read: d_ij (i < j)
 *           at D[j * n + i]; a pair with d_ij <= 0 counts as no pair (adds 0),
 *           like an unstored pair of fd_energy
 *   n       1 .. FD_NOALLOC_MAX_N; larger n returns FD_ERR_ARG
 *   dim     1..3
 *   f_out   host or device double; written with f(X)
 *   cuda_stream  stream to run on (NULL = legacy default); the call
 *           synchronises it before returning
 * All calls on a device share the scratch array: calls whose work overlaps on
 * the GPU (two streams, or two host threads at once) race and give wrong
 * results.  Every call looks up the array's address in the current device's
 * context (cudaGetSymbolAddress, which allocates nothing), so a device that
 * was reset gets the new address; the first call on a device also loads the
 * library's device code there, so make it before any stream capture.
 * Errors: FD_ERR_ARG (null pointer, X or D in host memory or on another
 * device, sizes out of range), FD_ERR_NONFINITE (the stress is not finite;
 * the value is still written), FD_ERR_CUDA. */
fd_status fd_energy_noalloc(const float* X, const float* D, int32_t n, int32_t dim, double* f_out,
                            void* cuda_stream);

/* Force F = (L^X - L^W) X = -(1/2) grad f(X) (Prop. 2.1 and Eq. (1)):
 * F_i = sum_{j != i} w_ij (d_ij / ||x_i - x_j|| - 1)(x_i - x_j); coincident
 * pairs contribute zero.  X and F_out are float32 [n][dim], host or device;
 * F_out is written.  Errors: FD_ERR_ARG, FD_ERR_NONFINITE, FD_ERR_CUDA. */
fd_status fd_forces(fd_layout* h, const float* X, float* F_out);

/* Largest graph accepted by fd_energy_length_grad and the adjoint's edge-
 * length derivative (fd_adjoint_reset / fd_adjoint_length_grad).  Up to 4096
 * vertices every source's search state sits in shared memory; above, in
 * 28 n bytes of device scratch per CTA (about 1.1 GB at the limit), beside
 * the float32 distance tiles and the tile array of pair sensitivities
 * (2 n^2 bytes each). */
#define FD_GRAD_MAX_N 131072

/* Derivative of the stress f(X) of Eq. (1) with respect to the edge lengths
 * of a weighted graph (d_ij = weighted shortest-path length, Sec. 2 and
 * Sec. 5.4; w_ij = d_ij^-2, Sec. 5.1).  With G_ij = d f / d d_ij =
 * -2 r_ij (r_ij - d_ij) / d_ij^3, the derivative for edge e is the sum of
 * G_ij over the pairs whose shortest path uses e; where two paths tie, the
 * path through the lower-index predecessor is used (ties have measure zero
 * for real-valued lengths).  The handle must come from fd_layout_create with
 * edge_len, on a connected simple graph (no self loops or repeated entries)
 * of at most FD_GRAD_MAX_N vertices.
 *   X         float32 [n][dim], host or device
 *   grad_len  float32[row_ptr[n]], host or device: one value per CSR entry,
 *             equal for the two entries of an undirected edge
 *   f_out     f(X) (host; may be NULL)
 * Errors: FD_ERR_ARG (handle without edge lengths, null pointers),
 * FD_ERR_UNIMPLEMENTED (n above the limit, disconnected or non-simple
 * graph), FD_ERR_NONFINITE, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_energy_length_grad(fd_layout* h, const float* X, float* grad_len, double* f_out);

/* Unrolled differentiation of Algorithm 2: the adjoint of one iteration.
 * The forward iteration (fd_sor_step) is b = L^X X (Prop. 2.1), Y solving
 * L^W Y = b with vertex 0 pinned (Eq. (2-5), Sec. 2), and X' = (1 + omega) Y -
 * omega X if line 6 kept the extrapolation (Eq. (10)), else X' = Y.  Given
 * Xbar_k1 = dL/dX' this writes Xbar_k = dL/dX with the acceptance held fixed:
 * the pinning's adjoint, one solve L^W lam = Ybar by the layout kernel's CG
 * (opt->cg_tol, opt->cg_max, opt->solver; NULL = defaults), and the transposed Jacobian
 * of L^X X applied to lam.  After fd_adjoint_reset, it also adds every pair's
 * sensitivity dL/dd_ij to an accumulator of the handle (weighted graphs that
 * fd_energy_length_grad accepts); fd_adjoint_length_grad turns the sum into
 * dL/dl_e through the shortest paths.
 *   X_k, X_k1   float32 [n][dim]: the iteration's input and output layouts
 *   accepted    the outcome of line 6 (fd_sor_step's *accepted)
 *   omega       the omega the iteration used (times the per-vertex factors of
 *               fd_set_vertex_omega, if set, as in the forward iteration)
 *   Xbar_k1     float32 [n][dim]: dL/dX_k1;  Xbar_k: float32 [n][dim], written
 *   cg_steps    CG steps of the adjoint solve (host; may be NULL)
 * Arrays host or device.  Errors: FD_ERR_ARG, FD_ERR_NONFINITE, FD_ERR_CUDA,
 * FD_ERR_TIMEOUT. */
fd_status fd_sor_step_adjoint(fd_layout* h, const float* X_k, const float* X_k1, int32_t accepted, double omega,
                              const float* Xbar_k1, float* Xbar_k, const fd_options* opt, int32_t* cg_steps);

/* Clears (allocating on first use) the handle's accumulator of pair
 * sensitivities.  Weighted graphs only, with the limits of
 * fd_energy_length_grad.  Errors: FD_ERR_ARG (no edge lengths),
 * FD_ERR_UNIMPLEMENTED, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_adjoint_reset(fd_layout* h);

/* dL/dl_e from the accumulated pair sensitivities (the sum over the
 * fd_sor_step_adjoint calls since fd_adjoint_reset), pushed through every
 * pair's shortest path as in fd_energy_length_grad; float32[row_ptr[n]],
 * host or device, equal for the two entries of an edge.  Errors: FD_ERR_ARG
 * (no accumulator), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_adjoint_length_grad(fd_layout* h, float* grad_len);

/* One iteration of Algorithm 2 (lines 4-8): H step by CG on Eq. (2-5) with
 * the first vertex pinned at the origin, extrapolation Eq. (10) with the
 * omega the strategy gives for iteration index k (k >= 0), acceptance test
 * of line 6 (ties accept).  X (float32 [n][dim], host or device) holds X^k
 * on entry and the accepted X^{k+1} on return.
 *   f_out      f(X^{k+1}) (host; may be NULL)
 *   accepted   1 if the extrapolated layout was kept (host; may be NULL)
 *   crit_out   termination criterion of opt->stop (host; may be NULL)
 * Errors: FD_ERR_ARG, FD_ERR_NONFINITE, FD_ERR_CG_BREAKDOWN, FD_ERR_TIMEOUT,
 * FD_ERR_CUDA. */
fd_status fd_sor_step(fd_layout* h, float* X, const fd_options* opt, int32_t k, double* f_out,
                      int32_t* accepted, double* crit_out);

/* Direct solver of Eq. (2-5).  L^W does not change during a run, so its
 * factorisation is made once (Sec. 2 names Cholesky factorisation for this
 * system).  fd_factor builds, in device memory, the dense FP32 inverse of
 *     A' = L^W + (sigma / n) 1 1^T,   sigma = (1/n) sum_i s_i,
 * (Gauss-Jordan elimination in 128 x 128 blocks, no pivoting: A' is positive
 * definite).  A' has the eigenvalues of L^W except that the null vector 1
 * gets sigma, so its condition number is that of L^W, not the n-fold one of
 * the pinned matrix; for a right-hand side of zero sum A'^-1 b solves
 * L^W z = b, and pinning vertex 0 is a translation.  With
 * opt->solver = FD_SOLVER_DIRECT every H step then refines from the warm
 * start: x += A'^-1 r, r -= L^W (A'^-1 r), until opt->cg_tol or opt->cg_max.
 * Memory: 4 n_pad^2 bytes (n_pad = n rounded up to 128), kept by the handle
 * until fd_factor_release or destroy.  Cost: about 2 n_pad^3 FP32 flops.
 *   n   at most FD_DIRECT_MAX_N
 * Errors: FD_ERR_ARG (n too large), FD_ERR_OOM, FD_ERR_CG_BREAKDOWN (a pivot
 * was not positive: the matrix is not numerically positive definite in FP32),
 * FD_ERR_CUDA. */
#define FD_DIRECT_MAX_N 32768
fd_status fd_factor(fd_layout* h);

/* Rows row0 .. row0 + nrows - 1 of A'^-1 (columns 0 .. n - 1), as float64 to
 * the host array out[nrows][n].  Errors: FD_ERR_ARG (not factored, range),
 * FD_ERR_CUDA. */
fd_status fd_factor_rows(fd_layout* h, int32_t row0, int32_t nrows, double* out);

/* Frees the inverse made by fd_factor.  Errors: FD_ERR_ARG. */
fd_status fd_factor_release(fd_layout* h);

/* Per-vertex relaxation factors (Sec. 6, first item of further work: a
 * separate stride factor for every vertex, x~_i = x_i^{k+1} + omega_i
 * (x_i^{k+1} - x_i^k)).  Every later fd_run / fd_sor_step of the handle uses
 * omega_i = omega m_i, omega being the factor the strategy gives for the
 * iteration; FD_OMEGA_FIXED with omega = 1 makes m the paper's omega vector.
 * The acceptance test (line 6 of Algorithm 2) is unchanged.  With
 * FD_OMEGA_ENUM the candidates are x + omega_e m (x - x_prev).
 *   m   float32 [n] (host or device), every m_i finite and >= 0; copied.
 *       NULL restores omega_i = omega.
 * Errors: FD_ERR_ARG (negative or non-finite factor), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_set_vertex_omega(fd_layout* h, const float* m);

/* Algorithm 2 from X^0 (omega = 0 with FD_OMEGA_FIXED is Algorithm 1) until
 * the termination rule holds or opt->max_iter iterations ran.  The whole
 * loop runs on the GPU in one cooperative launch; nothing returns to the
 * host between iterations.  X (float32 [n][dim], host or device) holds X^0
 * on entry and the final layout on return.
 *   iters_out  iterations performed (host; may be NULL)
 *   f_out      final stress (host; may be NULL)
 *   trace_f    NULL or host double[max_iter + 1]: f(X^0), f(X^1), ...
 * Errors: as fd_sor_step. */
fd_status fd_run(fd_layout* h, float* X, const fd_options* opt, int32_t* iters_out,
                 double* f_out, double* trace_f);

/* Per-iteration trace of the last fd_run, copied to host arrays of length
 * >= iterations (any pointer may be NULL): accepted flags, omega used,
 * CG steps and termination criterion of each iteration. */
fd_status fd_run_trace(fd_layout* h, int32_t* accepted, double* omega, int32_t* cg_steps,
                       double* crit);

/* More of the last fd_run / fd_sor_step's per-iteration trace, to host
 * arrays of length >= iterations (any pointer may be NULL): f(H(X^k)) (the
 * omega = 0 candidate of line 4), f of the extrapolated candidate of line 5
 * (under FD_OMEGA_ENUM the argmin), and the device time in ms from the
 * start of the launch to the end of each iteration (%globaltimer). */
fd_status fd_run_trace_ext(fd_layout* h, double* f_h, double* f_extrapolated, double* t_ms);

/* Ideal distances of rows row0 .. row0 + nrows - 1 (all n columns, d_ii = 0)
 * as stored by the handle, written as float64 to the host array
 * out[nrows][n].  Unit-edge graphs give exact integers.  Errors: FD_ERR_ARG,
 * FD_ERR_CUDA. */
fd_status fd_distance_rows(fd_layout* h, int32_t row0, int32_t nrows, double* out);

/* Facts about the handle (host struct). */
fd_status fd_layout_info(const fd_layout* h, fd_info* info);

/* Statistics of the last call on the handle (host struct). */
fd_status fd_last_stats(const fd_layout* h, fd_stats* stats);

/* Measured FP32 FMA throughput of the current device (the denominator of
 * the layout kernel's roofline, beside the nominal SMs x 128 lanes x 2 flop
 * x clock): every thread runs 16 independent FMA chains, scalar
 * (packed = 0, fma.rn.f32) or two-wide (packed = 1, fma.rn.f32x2, the
 * instruction the pair passes use); best of 5 timed launches.
 *   tflops  TFLOP/s (host)        ms  the best launch's time (host)
 * Errors: FD_ERR_ARG, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_fp32_peak(int32_t packed, double* tflops, double* ms);

/* Phase timeline (tracing).  fd_timeline_enable(h, cap) makes every later
 * layout-kernel launch record, at each of its grid-wide barriers, the
 * device time (ns since the launch started, from %globaltimer) and a phase
 * tag: 1 pack, 2 stress pass, 3 force pass, 4 initial RHS pass, 5 H-step
 * start (L^W x0), 6 L^W u0, 7 CG step (or L^W of a refinement step),
 * 8 stress/RHS of the candidates, 9 per-row-block reduction and vector
 * update after a pass, 10 application of the factored inverse.
 * cap = 0 disables it.  fd_timeline_read copies up to cap entries of the
 * last launch (tags and times as doubles, interleaved: tag, t, tag, t, ...)
 * and the number recorded.  Errors: FD_ERR_ARG, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_timeline_enable(fd_layout* h, int32_t cap);
fd_status fd_timeline_read(fd_layout* h, double* out, int32_t cap, int32_t* count);

/* ------------------------------------------------------------------------
 * Batched form: many independent small graphs laid out in one persistent
 * kernel launch.  Each graph runs the same Algorithm 2 as fd_run (H step by
 * CG on Eq. (2-5), extrapolation Eq. (10), acceptance test of line 6, the
 * termination rule of fd_stop_rule) and stops on its own criterion; graphs
 * share nothing but the launch.
 * ------------------------------------------------------------------------ */

typedef struct fd_batch fd_batch; /* opaque; owns every graph's distances and state */

/* Largest graph of a batch (vertices). */
#define FD_BATCH_MAX_N 2048

/* Size buckets of the tile-edge choice: bucket k holds the graphs with
 * 32 * 2^(k-1) < n <= 32 * 2^k (bucket 0: n <= 32; bucket 6: n <= 2048). */
#define FD_BATCH_BUCKETS 7

/* Facts about a batch handle. */
typedef struct {
  int32_t num_graphs, dim;
  int64_t total_vertices;  /* sum of the graphs' n */
  int64_t num_tiles;       /* stored 128 x 128 tiles over all graphs */
  int64_t distance_bytes;  /* device bytes of the uint8 distance tiles */
  int32_t max_n;           /* largest graph */
  int32_t max_diameter;    /* largest stored d_ij over all graphs (fill included) */
  int32_t disconnected;    /* graphs with unreachable pairs (filled under policy 1) */
  int32_t sm_count;
  int32_t grid;            /* CTAs of the persistent kernel */
  int32_t groups;          /* 128-thread tile groups per CTA (1 or 2) */
  int32_t stages;          /* tiles in flight per group (2 or 3) */
  int32_t graph_captured;  /* 1 once the launch runs from a captured CUDA graph */
  double apsp_ms;          /* device time of the batched shortest-path kernels at creation */
  int64_t small_tile_bytes;  /* device bytes of the 32 x 32 and 64 x 64 tiles (graphs below tile edge 128) */
  int32_t graphs_t128, graphs_t64, graphs_t32;  /* graphs laid out at tile edge 128, 64, 32 */
} fd_batch_info;

/* Builds a batch of num_graphs undirected graphs in one concatenated CSR:
 * graph g owns vertices graph_ptr[g] .. graph_ptr[g+1] - 1 (0-based,
 * graph_ptr[0] = 0) and every edge of the CSR joins two vertices of the
 * same graph.  Each graph has 1 .. FD_BATCH_MAX_N vertices.  Computes every
 * graph's hop distances (bit-parallel BFS, one 64-source batch per CTA) and
 * the row sums of its L^W; unit edge lengths only, hop diameter (fill
 * included) at most 253.
 *   graph_ptr  int32[num_graphs + 1], host or device
 *   row_ptr    int32[N + 1] with N = graph_ptr[num_graphs], host or device
 *   col_idx    int32[row_ptr[N]] global vertex ids, host or device
 *   disconnected_policy, cuda_stream: as in fd_layout_create
 * Errors: FD_ERR_ARG (sizes, a graph above FD_BATCH_MAX_N), FD_ERR_CSR
 * (malformed, non-symmetric, or an edge between graphs), FD_ERR_DISCONNECTED,
 * FD_ERR_UNIMPLEMENTED (a diameter above 253), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_batch_create(fd_batch** out, int32_t num_graphs, int32_t dim, const int32_t* graph_ptr,
                          const int32_t* row_ptr, const int32_t* col_idx, int32_t disconnected_policy,
                          void* cuda_stream);

/* Releases every resource of the batch (NULL is a no-op). */
void fd_batch_destroy(fd_batch* b);

/* Algorithm 2 on every graph of the batch, in one persistent launch per tile
 * edge in use (the graphs at edge 128, 64 and 32 in turn, all three replayed
 * from one captured CUDA graph after the first call with the same launch
 * configuration).  X (float32 [N][dim], host or device; graph g's rows are
 * graph_ptr[g] ..) holds every X^0 on entry and the final layouts on return.
 *   opt        strategy FD_OMEGA_FIXED or FD_OMEGA_PROB (the same omega
 *              sequence for every graph); FD_OMEGA_ENUM and FD_SOLVER_DIRECT
 *              return FD_ERR_UNIMPLEMENTED (the batched kernel solves by CG).
 *              tol, stop, max_iter, cg_tol, cg_max apply to every graph.
 *   omega      NULL (every graph uses opt->omega) or double[num_graphs]
 *              (host or device): graph g's fixed omega (FD_OMEGA_FIXED)
 *   iters      NULL or host int32[num_graphs]: iterations per graph
 *   f_out      NULL or host double[num_graphs]: final stress per graph
 * Per-graph failures (non-finite input or stress) are reported by
 * fd_batch_results and make the call return FD_ERR_NONFINITE after every
 * other graph has finished.  Errors: FD_ERR_ARG, FD_ERR_UNIMPLEMENTED,
 * FD_ERR_NONFINITE, FD_ERR_TIMEOUT, FD_ERR_CUDA. */
fd_status fd_batch_run(fd_batch* b, float* X, const fd_options* opt, const double* omega, int32_t* iters,
                       double* f_out);

/* Per-graph details of the last fd_batch_run, to host arrays of length
 * num_graphs (any pointer may be NULL): fd_status of the graph, CG steps,
 * accepted extrapolations, last termination criterion, L^W passes, stress
 * passes (per candidate), and the device time (ms, %globaltimer) the CTA
 * that ran the graph spent on it. */
fd_status fd_batch_results(const fd_batch* b, int32_t* status, int32_t* cg_steps, int32_t* accepted, double* crit,
                           double* matvec_passes, double* stress_passes, double* graph_ms);

/* The autotuner.  Times `probe_iter` iterations of Algorithm 2 from X (host
 * or device, left unchanged), best of `repeats` runs each:
 *   1. the launch shape: 128-thread units per CTA in {1, 2} x tiles in
 *      flight per tile group in {2, 3}, on every graph;
 *   2. then, size bucket by bucket (FD_BATCH_BUCKETS), the tile edge
 *      T in {128, 64, 32} of that bucket's graphs, each bucket's graphs run
 *      alone.  A graph at edge T is cut into ceil(n / T) blocks and T x T
 *      tiles, computed by groups of T threads.
 * The winners are kept for later runs (*groups and *stages receive the
 * shape, fd_batch_get_tiles the edges) and the edges are stored in a
 * process-wide cache per (bucket, dim) from which fd_batch_create starts
 * later batches of the same dimension.  Errors: as fd_batch_run. */
fd_status fd_batch_tune(fd_batch* b, const float* X, const fd_options* opt, int32_t probe_iter, int32_t repeats,
                        int32_t* groups, int32_t* stages);

/* Sets the launch shape directly (groups 1 or 2, stages 2 or 3).
 * Errors: FD_ERR_ARG (infeasible shape). */
fd_status fd_batch_set_shape(fd_batch* b, int32_t groups, int32_t stages);

/* Sets the tile edge of each size bucket directly: tiles is a host
 * int32[FD_BATCH_BUCKETS] of 32, 64 or 128 (the graphs of bucket k are laid
 * out at edge tiles[k]); re-tiles the affected graphs' distance codes on the
 * device.  Errors: FD_ERR_ARG (another value), FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_batch_set_tiles(fd_batch* b, const int32_t* tiles);

/* The tile edge of each size bucket, to a host int32[FD_BATCH_BUCKETS]. */
fd_status fd_batch_get_tiles(const fd_batch* b, int32_t* tiles);

/* The process-wide cache of tuned tile edges for layout dimension dim (1-3),
 * to a host int32[FD_BATCH_BUCKETS] (0 = bucket not tuned yet), and its reset.
 * fd_batch_create gives an untuned bucket edge 128. */
fd_status fd_batch_cached_tiles(int32_t dim, int32_t* tiles);
void fd_batch_clear_tile_cache(void);

/* The hop distances of graph g as stored, float64 [n_g][n_g] host array
 * (d_ii = 0).  Errors: FD_ERR_ARG, FD_ERR_OOM, FD_ERR_CUDA. */
fd_status fd_batch_distances(fd_batch* b, int32_t g, double* out);

/* Facts about the batch; statistics of its last run (sums over graphs:
 * iterations, cg_steps, accepted, pair_passes weighted by each graph's
 * pairs in `pairs` = sum over graphs of pair_passes_g * n_g (n_g - 1) / 2,
 * kernel_ms of the one launch). */
fd_status fd_batch_get_info(const fd_batch* b, fd_batch_info* info);
fd_status fd_batch_last_stats(const fd_batch* b, fd_stats* stats);

/* Status of the last failing call on the handle (FD_OK if none). */
fd_status fd_last_error(const fd_layout* h);

/* Static, human-readable name of a status code. */
const char* fd_status_string(fd_status s);

#ifdef __cplusplus
}
#endif

#endif /* FD_LAYOUT_H */
