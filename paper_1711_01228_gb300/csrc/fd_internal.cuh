// fd_internal.cuh -- shared definitions of the CUDA layout engine.
//
// Geometry.  Vertices are padded to n_pad = nb * TILE.  The unordered pairs
// of tile blocks are covered by a "half ring": block row I owns the tiles
// (I, J) with J = (I + k) mod nb for k = 0 .. L_I - 1, where
//   L_I = (nb + 1) / 2                    if nb is odd,
//   L_I = nb / 2 + 1 (I < nb/2), nb / 2   if nb is even.
// Every unordered block pair appears exactly once and every block row owns
// about nb/2 tiles, so both the rows and the per-row-block reductions (about
// nb/2 column partials each) are balanced.  Tile k = 0 is the diagonal block,
// which holds only the pairs i < j.
//
// A tile stores one code per (i, j) pair, column-major over i: byte
// [jl * TILE + il] for i = I*TILE + il, j = J*TILE + jl.  Code 0 means "no
// pair" (padding, i >= j inside a diagonal tile).  A real pair stores its
// ideal distance d_ij as a uint8 hop count, or as float32 1/d_ij (the
// correctly rounded reciprocal): the pair loop needs 1/d and 1/d^2, and the
// reciprocal spares it a division per pair; an unreached pair (0) stays 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdl {

constexpr int TILE = 128;          // vertices per tile side
constexpr int CTA = 128;           // threads per CTA of the pair kernels (4 warps)
constexpr int LUT_N = 256;         // uint8 codes
constexpr int LUT_ROW = 256;       // bytes per code in the replicated table: 32 x 1/d, then 32 x 1/d^2
constexpr int SC_STRIDE = 36;      // scalars of one grid-wide reduction, at most
constexpr int MAX_NBUF = 4;        // stages of the tile pipeline
constexpr int MAX_CTA_TASKS = 128; // task descriptors a CTA keeps in shared memory

enum CodeKind { CODE_U8 = 0, CODE_F32 = 1 };

// Modes of the cooperative kernel.
// KM_SOLVE: one H-step solve of L^W Y = B for a given B (x_in), Y pinned at
// vertex 0 (the adjoint of Eq. (2-5) needs it with another right-hand side).
enum KernelMode { KM_ENERGY = 0, KM_FORCES = 1, KM_RUN = 2, KM_SOLVE = 3 };

// Error codes shared with fd_status (include/fd_layout.h).
enum {
  E_OK = 0,
  E_NONFINITE = 4,
  E_CG_BREAKDOWN = 5,
  E_TIMEOUT = 7,
};

// A run of consecutive tiles of one strip.  Every CTA owns a contiguous
// range of the strip-major tile order (the same number of tiles, +-1, for
// every CTA), cut into tasks at strip boundaries.
struct TaskDesc {
  int I;      // block row
  int k0;     // first tile offset in the strip
  int k1;     // one past the last tile offset
  int tile0;  // global index of tile (I, k0)
};

// Device control block of one cooperative launch.
struct Ctrl {
  unsigned long long reserved0;
  unsigned int bar_count;      // grid barrier arrivals
  unsigned int bar_gen;        // grid barrier generation
  int err;                     // first error (0 = none)
  int iters;                   // outer iterations done
  int cg_steps;                // CG steps over the launch
  int cg_maxed;                // H solves stopped by cg_max
  int accepted;                // extrapolations kept
  int cg_stalled;              // CG columns stopped early because the curvature estimate lost positivity
  double f_final;              // stress of the output layout
  double crit_final;           // last termination criterion
  double pair_passes;          // all-pairs passes evaluated
  double matvec_passes;        // y = L^W p passes
  double stress_passes;        // stress (+ RHS or force) passes, per candidate
  double enum_passes;          // candidate stresses of the enumerating strategy (NENUM per enumeration pass)
  double rhs_skipped;          // candidate evaluations (in stress_passes) without their right-hand side
  int timeout_where;           // barrier index that timed out (diagnostic)
  int timeline_n;              // timeline entries written
  unsigned long long t_start;  // %globaltimer at kernel start (CTA 0)
  float2 red[SC_STRIDE];       // grid-wide sums of a reduction barrier (double-float), written by its last CTA
  double red_d[4];             // FP64 scalars computed by that CTA (termination criterion)
  // every CTA adds its partial sums (FP64 atomics) to set (b & 1) before it
  // arrives at reduction barrier b; the last CTA at barrier b clears set
  // (b + 1) & 1, read after barrier b - 1, for the next reduction
  double acc_d[2][SC_STRIDE];
};

struct Geometry {
  int n, n_pad, nb, dim;
  int ntiles, ntasks;
  const int* tile_base;        // [nb + 1] first tile index of each strip
  const int* strip_len;        // [nb] L_I
  const TaskDesc* tasks;       // [ntasks], grouped by CTA
  const int* cta_task_ptr;     // [grid + 1] CTA b runs tasks cta_task_ptr[b] .. cta_task_ptr[b+1]-1
};

// Parameters of the cooperative kernel (passed by value).
enum Solver { SOLVER_CG = 0, SOLVER_DIRECT = 1 };

struct KParams {
  Geometry g;
  int mode;
  const void* D;               // distance tiles
  const unsigned char* lut;    // [lut_rows][LUT_ROW] replicated table: 32 x 1/d, then 32 x 1/d^2
  int lut_rows;                // codes 0 .. lut_rows-1 present in the tiles
  int nbuf;                    // stages of the tile pipeline (2 to 4)
  int tps;                     // tiles per stage (1, or 2 consecutive tiles of a task)
  const float* s;              // [n_pad] row sums of W (diagonal of L^W)
  const float* inv_s;          // [n_pad] 1/s (0 for padding)
  const float* x_in;           // [n][dim] input layout (device staging)
  float* x_out;                // [n][dim] output (layout or forces)
  // internal vectors, [n_pad][DIMP] with DIMP = 1, 2, 4 for dim = 1, 2, 3:
  // layout X^k and the H step's right-hand side B = L^{X^k} X^k and initial
  // residual R0 = B - L^W X^k; Xt, Bz, Bt spare; CG state Zw (iterate),
  // R (residual), U = M^-1 R, W = L^W U, P, S = L^W P
  float *X, *R0, *Xt, *B, *Bz, *Bt, *Zw, *R, *U, *W, *P, *S;
  // per-vertex sums of a pass, [3][n_pad][DIMP] FP64: the pair kernels add
  // their FP32 row and column partial sums with FP64 atomics; the vertex phase
  // after the pass reads them and clears them for the next pass
  double* acc;
  Ctrl* ctrl;
  const double* omega_seq;     // [max_iter] omega of each iteration
  double* trace_f;             // [max_iter + 1]
  int* trace_acc;              // [max_iter]
  double* trace_om;            // [max_iter]
  int* trace_cg;               // [max_iter]
  double* trace_crit;          // [max_iter]
  double* trace_fh;            // [max_iter] f(H(X^k)) (the omega = 0 candidate)
  double* trace_ft;            // [max_iter] f of the extrapolated candidate (the argmin under enumeration)
  double* trace_t;             // [max_iter] ms since the launch began, at the end of iteration k
  int max_iter, stop, cg_max;
  int enum_omega;              // 1: omega is the argmin of f over {0, 0.5, ..., 9} each iteration (Sec. 5.2.2)
  const float* om_scale;       // NULL, or [n_pad] per-vertex factors m_i: omega_i = omega m_i (Sec. 6), padding 0
  // direct solver: the H step refines with A'^-1 = (L^W + sigma/n 1 1^T)^-1
  // ([n_pad][n_pad], row-major) in place of CG
  const float* ainv;
  int solver;                  // SOLVER_CG or SOLVER_DIRECT
  double tol, cg_tol;
  long long timeout_ns;        // limit of every mbarrier (copy) wait
  long long bar_timeout_ns;    // limit of every grid-barrier wait
  double* timeline;            // NULL, or [timeline_cap][2] {tag, ns} written by CTA 0 at each barrier
  int timeline_cap;
};

// ------------------------------------------------------------------------
// Batched form: many independent graphs, each with its own half ring
// ------------------------------------------------------------------------

constexpr int BMAX_N = 2048;  // largest graph of the batched form

// Half-ring geometry of an nb-block graph: strip length and first tile of
// block row I (the same layout as above, in closed form).
__host__ __device__ __forceinline__ int hr_len(int nb, int I) {
  return (nb & 1) ? (nb + 1) / 2 : (I < nb / 2 ? nb / 2 + 1 : nb / 2);
}
__host__ __device__ __forceinline__ int hr_base(int nb, int I) {
  if (nb & 1) return I * ((nb + 1) / 2);
  const int h = nb / 2;
  return (I <= h) ? I * (h + 1) : h * (h + 1) + (I - h) * h;
}
__host__ __device__ __forceinline__ int hr_tiles(int nb) { return nb * (nb + 1) / 2; }

// One graph of a batch.
struct BGraph {
  int n, nb;     // vertices, blocks of TILE vertices
  int v0;        // first vertex of the graph in the caller's concatenated arrays
  int p0;        // first padded vertex in the internal pools (a multiple of TILE)
  long long t0;  // first tile of the graph in the distance pool (TILE x TILE tiles)
  // tile edge of the layout kernel: T = TILE reads the tiles at t0; T = 32 or
  // 64 reads nbt = ceil(n / T) blocks' half ring of T x T tiles (the same
  // layout at the smaller edge) from byte dt of the small-tile pool
  int T, nbt;
  long long dt;
};

// Parameters of one batched launch (device memory, so that a captured CUDA
// graph keeps one pointer while the host rewrites the block between runs).
struct BParams {
  const BGraph* graphs;   // [G]
  const int* order;       // [G] processing order: the graphs of tile class 0, 1, 2 (T = 128, 64, 32), each largest first
  int cls_off[4];         // class c owns order[cls_off[c] .. cls_off[c + 1])
  int G, dim;
  const unsigned char* D; // uint8 distance tiles of every graph (TILE x TILE)
  const unsigned char* DT;// the graphs with T < TILE: their T x T tiles
  const unsigned char* lut;
  int lut_rows;
  const float* s;         // [P] row sums of W (diagonal of L^W)
  const float* inv_s;     // [P] 1 / s (0 for padding)
  const float* x_in;      // [N][dim] input layouts, concatenated
  float* x_out;           // [N][dim] output layouts
  float *X, *Z, *R, *Pd, *B;  // [P][DP] layout, CG iterate, residual, direction, right-hand side
  float* R0;              // [P][DP] the next H step's starting residual (between refresh passes)
  const double* omega;    // [G] omega of each graph (FD_OMEGA_FIXED)
  const double* omega_seq;// [max_iter] omega of iteration k (FD_OMEGA_PROB), or NULL
  int max_iter, cg_max, stop;
  double tol, cg_tol;
  int* queue;             // [3] next position of each tile class in its part of `order`
  int* err;               // first launch-level error
  // per-graph results
  int* iters;
  int* cg_steps;
  int* accepted;
  int* status;
  double* f_final;
  double* crit_final;
  double* passes_mv;      // [G] L^W passes
  double* passes_st;      // [G] stress passes (per candidate)
  double* graph_ms;       // [G] device time the CTA spent on the graph
  int nbuf;
  int n_pad_max;
  long long timeout_ns;
};

// ------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// Every wait is bounded: after timeout_ns the CTA records E_TIMEOUT and
// leaves.  Returns false if an error is pending (the caller must return).
__device__ __forceinline__ bool grid_sync(Ctrl* c, long long timeout_ns, int where) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &c->bar_gen;
    volatile int* err = &c->err;
    unsigned int g = *gen;
    __threadfence();
    unsigned int arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned long long t0 = globaltimer_ns();
      unsigned int ns = 32;
      while (*gen == g) {
        if (*err != 0) break;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
          atomicCAS(&c->err, 0, (int)E_TIMEOUT);
          atomicExch(&c->timeout_where, where);
          break;
        }
      }
    }
    __threadfence();
    s_ok = (*err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void set_error(Ctrl* c, int code) { atomicCAS(&c->err, 0, code); }

// Tracing: CTA 0, thread 0 appends (tag, ns since launch) to the timeline.
__device__ __forceinline__ void tl_mark(const KParams& p, int tag) {
  if (p.timeline && blockIdx.x == 0 && threadIdx.x == 0 && p.ctrl->timeline_n < p.timeline_cap) {
    const int q = p.ctrl->timeline_n++;
    p.timeline[2 * q] = (double)tag;
    p.timeline[2 * q + 1] = (double)(globaltimer_ns() - p.ctrl->t_start);
  }
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Kahan-compensated accumulation.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
  float y = v - comp;
  float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// shared-memory mbarrier + 1-D bulk copy (TMA) helpers
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders this thread's view of generic-proxy global writes (made visible by a
// grid barrier) before its subsequent bulk-copy (async-proxy) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Both of the above: before a bulk copy that overwrites shared memory just
// read by this CTA and reads global memory written before a grid barrier.
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
  }
  return true;
}

}  // namespace fdl
