// fd_solver.cuh -- the cooperative layout kernel (stress, forces, and the
// whole Algorithm 2 loop of Wang & Wang 2012) for one layout dimension and
// one distance-code type.  Included by fd_solver_d{1,2,3}.cu.
//
// Work decomposition
// ------------------
// All-pairs passes run over the tiles of the half ring (fd_internal.cuh),
// grouped into tasks of consecutive tiles of one block row.  CTA b takes
// tasks b, b + G, b + 2G, ... (G CTAs), in reverse order on every other pass
// so that the tiles one pass reads last are still in L2 when the next starts.
//
// Inside a tile (128 x 128 pairs) every lane holds R consecutive rows of
// block I (R = 16 for L^W products, 8 for the stress / right-hand-side
// passes; half that in 3-D) and a group of G = 128 / R lanes covers all 128
// rows; the R groups of the CTA take G columns of block J each.  In step t
// lane q of a group pairs its rows with column (q + t) mod G of the group, so
// after G steps both endpoints of every pair have been accumulated exactly
// once (symmetric n-body); the column sums are gathered from the lanes with
// shuffles.  Two rows share one packed FP32x2 instruction.  1/d and 1/d^2
// come from a table in shared memory replicated per lane (one bank each),
// addressed by one byte permute of the code word.
//
// Pipeline: a tile's distance codes (16 KB for uint8) and the raw per-vertex
// arrays of block J (and of block I at the first tile of a task) arrive by
// 1-D bulk copies (TMA) on an mbarrier, nbuf - 1 tiles ahead.  The raw
// arrays are turned into the pass's vectors in place in shared memory (e.g.
// the CG vector u = M^-1 (r - alpha s) is formed on the fly).
//
// Reductions: the column sums of a tile and the row sums of a task are added
// to per-vertex accumulators with FP32 vector atomics (order-dependent in
// the last bits).  After the pass (grid barrier) a vertex phase, one thread
// per vertex, reads and clears the accumulators and runs the step's
// per-vertex work.  Scalars (stress, CG dot products, displacement sums) are
// double-float numbers: per-CTA partial sums, reduced in a fixed order once
// by the last CTA to reach the next grid barrier.
#pragma once

#include "fd_internal.cuh"

namespace fdl {

template <int DIM>
struct DimP {
  static constexpr int v = (DIM == 3) ? 4 : DIM;
};

template <int DIM>
struct Vec {
  float c[DIM];
};

template <int DIM>
__device__ __forceinline__ Vec<DIM> ldv(const float* a, int i) {
  Vec<DIM> r;
  if constexpr (DIM == 1) {
    r.c[0] = __ldcg(a + i);
  } else if constexpr (DIM == 2) {
    float2 t = __ldcg(reinterpret_cast<const float2*>(a) + i);
    r.c[0] = t.x;
    r.c[1] = t.y;
  } else {
    float4 t = __ldcg(reinterpret_cast<const float4*>(a) + i);
    r.c[0] = t.x;
    r.c[1] = t.y;
    r.c[2] = t.z;
  }
  return r;
}

template <int DIM>
__device__ __forceinline__ void stv(float* a, int i, const Vec<DIM>& v) {
  if constexpr (DIM == 1) {
    __stcg(a + i, v.c[0]);
  } else if constexpr (DIM == 2) {
    __stcg(reinterpret_cast<float2*>(a) + i, make_float2(v.c[0], v.c[1]));
  } else {
    __stcg(reinterpret_cast<float4*>(a) + i, make_float4(v.c[0], v.c[1], v.c[2], 0.f));
  }
}

template <int DIM>
__device__ __forceinline__ Vec<DIM> lds_v(const float* a, int i) {
  Vec<DIM> r;
  if constexpr (DIM == 1) {
    r.c[0] = a[i];
  } else if constexpr (DIM == 2) {
    float2 t = reinterpret_cast<const float2*>(a)[i];
    r.c[0] = t.x;
    r.c[1] = t.y;
  } else {
    float4 t = reinterpret_cast<const float4*>(a)[i];
    r.c[0] = t.x;
    r.c[1] = t.y;
    r.c[2] = t.z;
  }
  return r;
}
template <int DIM>
__device__ __forceinline__ void sts_v(float* a, int i, const Vec<DIM>& v) {
  if constexpr (DIM == 1) {
    a[i] = v.c[0];
  } else if constexpr (DIM == 2) {
    reinterpret_cast<float2*>(a)[i] = make_float2(v.c[0], v.c[1]);
  } else {
    reinterpret_cast<float4*>(a)[i] = make_float4(v.c[0], v.c[1], v.c[2], 0.f);
  }
}

template <int DIM>
__device__ __forceinline__ Vec<DIM> vzero() {
  Vec<DIM> v;
#pragma unroll
  for (int d = 0; d < DIM; ++d) v.c[d] = 0.f;
  return v;
}

// --------------------------------------------------------------------------
// Packed FP32x2 arithmetic: one instruction works on two rows.
// --------------------------------------------------------------------------
// (Packing and unpacking are register-pair moves, not arithmetic.)
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float lo2(f2x v) {
  float a;
  asm("{\n\t.reg .f32 hi;\n\tmov.b64 {%0, hi}, %1;\n\t}" : "=f"(a) : "l"(v));
  return a;
}
__device__ __forceinline__ float hi2(f2x v) {
  float b;
  asm("{\n\t.reg .f32 lo;\n\tmov.b64 {lo, %0}, %1;\n\t}" : "=f"(b) : "l"(v));
  return b;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Vector atomic add of one vertex's values to a per-vertex accumulator.
template <int DIM>
__device__ __forceinline__ void atomic_addv(float* a, int i, const Vec<DIM>& v) {
  if constexpr (DIM == 1) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(a + i), "f"(v.c[0]) : "memory");
  } else if constexpr (DIM == 2) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a + 2 * i), "f"(v.c[0]), "f"(v.c[1])
                 : "memory");
  } else {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a + 4 * i), "f"(v.c[0]),
                 "f"(v.c[1]), "f"(v.c[2]), "f"(0.f)
                 : "memory");
  }
}

// Per-vertex pass sums are FP64: every tile's FP32 column partial and every
// task's FP32 row partial are added to them with FP64 atomics, so the sum over
// the CTAs loses nothing to rounding and hardly depends on the order of the
// atomics (well below FP32 resolution, so runs repeat).  (No vector form of
// the FP64 reduction exists: one instruction per coordinate.)
template <int DIM>
__device__ __forceinline__ void atomic_addv(double* a, int i, const Vec<DIM>& v) {
  constexpr int DP = DimP<DIM>::v;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(a + (size_t)DP * i + d), "d"((double)v.c[d])
                 : "memory");
}

// Stores v (FP32) into accumulator entry i (a given right-hand side, or 0).
template <int DIM>
__device__ __forceinline__ void st_acc(double* a, int i, const Vec<DIM>& v) {
  constexpr int DP = DimP<DIM>::v;
#pragma unroll
  for (int d = 0; d < DIM; ++d) __stcg(a + (size_t)DP * i + d, (double)v.c[d]);
}

// PM_ENUM: stress of the NENUM extrapolations (1 + omega) z - omega x,
// omega = 0, 0.5, ..., 9, of one CG solution z (Sec. 5.2.2).
// PM_K2L: the two candidates' stresses and the right-hand side of the second
// only (the extrapolated layout, which line 6 of Algorithm 2 keeps in most
// iterations); when the first is kept, a PM_RHS pass of its own follows.
enum PairMode { PM_STRESS = 0, PM_FORCES = 1, PM_RHS = 2, PM_MATVEC = 3, PM_ENUM = 4, PM_K2L = 5 };
constexpr int NENUM = 19;
constexpr float ENUM_STEP = 0.5f;

// Stress sums of a pass: one per candidate, NENUM for PM_ENUM.
template <int MODE, int NC>
struct NStress {
  static constexpr int v = (MODE == PM_ENUM) ? NENUM : NC;
};

// How a pass forms its vectors from the raw arrays it copies.
enum SrcKind {
  SK_DIRECT = 0,  // v = a[0]
  SK_CGU = 1,     // u = inv_s * (r - alpha * (w + beta * s_prev)); a = {r, w, s_prev, inv_s}
  SK_K2 = 2,      // z = zw - z0 and (NC = 2) xt = (1 + omega) z - omega x; a = {zw, x}
  SK_SEL = 3,     // the candidate kept by line 6 of Algorithm 2: sel ? xt : z, from a = {zw, x}
  SK_ZX = 4       // z = zw - z0 and the previous layout x, from a = {zw, x}
};

// Raw arrays of a source kind.
__host__ __device__ constexpr int src_arrays(int kind) { return (kind == SK_DIRECT) ? 1 : (kind == SK_CGU) ? 4 : 2; }

struct PassSrc {
  int kind;  // SrcKind (a run-time value: one compiled pass serves every kind)
  const float* a[4];
  float alpha[3], beta[3];  // SK_CGU, per column
  float z0[3];              // SK_K2 / SK_SEL: vertex 0 of the CG solution (the pin of Sec. 2)
  float om;                 // SK_K2 / SK_SEL: omega of Eq. (10)
  int sel;                  // SK_SEL: 1 = the extrapolation was accepted
  const float* oms;         // SK_K2 / SK_SEL / SK_ZX: per-vertex factors m_i, omega_i = om * m_i (Sec. 6); NULL: all 1
};

// The CG vector u_{i+1} (used both on the fly and in the vertex phase, so
// that the two agree bit for bit).
__device__ __forceinline__ float cg_u(float r, float w, float sp, float is, float alpha, float beta) {
  return is * fmaf(-alpha, fmaf(beta, sp, w), r);
}
// Eq. (10): X~ = (1 + omega) X^{k+1} - omega X^k.
__device__ __forceinline__ float sor_xt(float z, float x, float om) { return fmaf(1.0f + om, z, -(om * x)); }

template <int CODE>
struct CodeBytes {
  static constexpr int v = (CODE == CODE_U8) ? 1 : 4;
};

// Bytes of one block (TILE vertices) of a pass's raw arrays.
template <int DIM>
__host__ __device__ constexpr int raw_bytes(int kind) {
  return (kind == SK_CGU) ? 3 * TILE * DimP<DIM>::v * 4 + TILE * 4 : src_arrays(kind) * TILE * DimP<DIM>::v * 4;
}

// Rows per lane and column-accumulator chains of a pass kind, for a tile of
// T x T pairs computed by T threads (T = TILE in the single-graph kernel; the
// batched kernel also runs T = 32 and 64).  G = T / R lanes cover the rows,
// and the T / G groups of G lanes take disjoint columns.  Chain h serves the
// steps t = h (mod CH) and travels CH lanes per use (no travel when CH = G).
template <int DIM, int MODE, int T = TILE>
struct TileShape {
  static constexpr int R = (MODE == PM_MATVEC) ? (DIM == 3 ? 8 : 16) : 4;
  static constexpr int G = T / R;
  static constexpr int CH0 = (MODE == PM_MATVEC) ? (DIM == 3 ? 4 : 8) : 2;
  static constexpr int CH = (CH0 < G) ? CH0 : G;
  static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "a column group is 2..32 lanes of one warp");
  static_assert(G % CH == 0, "chains must divide the group");
};

__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Shared memory: fixed part, the replicated lookup table (at a fixed offset,
// so that table reads need no address arithmetic: row c, 256 bytes, holds 32
// copies of 1/c (bytes 0..127) and 32 copies of 1/c^2 (bytes 128..255)),
// then nbuf pipeline stages (codes + raw arrays of blocks J and I).
template <int DIM, int CODE>
struct SmemLayout {
  static constexpr int DP = DimP<DIM>::v;
  static constexpr int DBUF = TILE * TILE * CodeBytes<CODE>::v;
  static constexpr int RAWB = align_up(raw_bytes<DIM>(SK_CGU), 128);
  static constexpr int OFF_RED64 = 0;     // float2 [CTA] reduction scratch
  static constexpr int OFF_MISC = 1024;   // mbarriers
  static constexpr int OFF_CTL = 1088;    // PassCtl of the running pass
  static constexpr int OFF_RUN = 1344;    // RunState of the Algorithm 2 loop
  static constexpr int OFF_PARAMS = 1536; // copy of the kernel parameters
  static constexpr int OFF_TASKS = 2048;  // this CTA's task descriptors
  static constexpr int OFF_LUT = OFF_TASKS + MAX_CTA_TASKS * 16;
  // A stage holds tps (1 or 2) consecutive tiles of a task: their codes, the
  // raw arrays of their column blocks (array-major: [array][tps][TILE][DP],
  // scalars [tps][TILE] after the vector arrays) and those of block I.
  __host__ __device__ static constexpr int stage(int tps) { return align_up(tps * DBUF + (tps + 1) * RAWB, 128); }
  __host__ __device__ static constexpr int stage_base(int lut_bytes) { return align_up(OFF_LUT + lut_bytes, 128); }
  __host__ __device__ static constexpr int off_d(int sb, int s, int tps) { return sb + s * stage(tps); }
  __host__ __device__ static constexpr int off_rawj(int sb, int s, int tps) { return sb + s * stage(tps) + tps * DBUF; }
  __host__ __device__ static constexpr int off_rawi(int sb, int s, int tps) {
    return sb + s * stage(tps) + tps * DBUF + tps * RAWB;
  }
  __host__ __device__ static constexpr int bytes(int nbuf, int lut_bytes, int tps) {
    return stage_base(lut_bytes) + nbuf * stage(tps);
  }
};

struct PairState {
  unsigned parity;  // bit b: phase parity of mbarrier b
  int pass;         // passes run so far (odd passes visit the tiles in reverse)
};

// What a pair pass needs from the kernel parameters (passed by value, so
// that the out-of-line pass keeps them in registers).
struct PassArgs {
  const void* D;
  const TaskDesc* tasks_g;  // this CTA's tasks in global memory
  const TaskDesc* tasks_s;  // ... and the first MAX_CTA_TASKS of them in shared memory
  Ctrl* ctrl;
  double* rsum;  // stress passes: the grid-wide sums (one per candidate) this CTA adds to
  long long timeout_ns;
  int n, n_pad, nb, ntasks, nbuf;  // ntasks: this CTA's
  int stage_base;                   // shared-memory offset of stage 0
  int tps;                          // tiles per stage (1 or 2)
};

// --------------------------------------------------------------------------
// Double-float reductions
// --------------------------------------------------------------------------

// Reductions use double-float numbers (hi + lo, each FP32, combined with the
// error-free TwoSum / TwoProduct transformations): about 44 significant bits
// at FP32 speed.  FP64 arithmetic is slow on this GPU and is kept to a few
// scalar operations per reduction.
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_of(float x) { return {x, 0.f}; }
// exact product of two floats
__device__ __forceinline__ df df_prod(float x, float y) {
  const float p = x * y;
  return {p, fmaf(x, y, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return {hi, e - (hi - s)};
}
// exact difference of two floats
__device__ __forceinline__ df df_diff(float x, float y) {
  const float s = x - y;
  const float bb = s - x;
  return {s, (x - (s - bb)) + (-y - bb)};
}
__device__ __forceinline__ df df_sqr(df a) { return df_add(df_prod(a.hi, a.hi), df_of(2.f * a.hi * a.lo)); }
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float df_f(df a) { return a.hi + a.lo; }
__device__ __forceinline__ df df_ld(const float2* p) {
  const float2 v = __ldcg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void df_st(float2* p, df a) { __stcg(p, make_float2(a.hi, a.lo)); }

// Sums K values over the CTA in a fixed order; the totals land in v[] of every thread.
template <int K>
__device__ __forceinline__ void cta_sum_multi(df (&v)[K], float2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df q;
      q.hi = __shfl_down_sync(0xffffffffu, v[k].hi, o);
      q.lo = __shfl_down_sync(0xffffffffu, v[k].lo, o);
      v[k] = df_add(v[k], q);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = make_float2(v[k].hi, v[k].lo);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    df t = {red[k].x, red[k].y};
#pragma unroll
    for (int w = 1; w < 4; ++w) t = df_add(t, df{red[w * K + k].x, red[w * K + k].y});
    v[k] = t;
  }
  __syncthreads();
}

// Grid barrier whose last arriving CTA runs `on_last(sums)` (all its
// threads) before it releases the others, with the grid-wide sums that the
// CTAs added before arriving.  Waits are bounded.
// Ordering: every CTA arrives with an acquire-release add on the counter
// (releasing its writes, which its threads ordered before thread 0 with the
// CTA barrier); the last arrival's add acquires all of them (the adds form
// one release sequence), and its release of the generation publishes them,
// with the reduction, to every CTA that acquires the new generation.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* a, unsigned int x) {
  unsigned int v;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "r"(x) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned int* a, unsigned int x) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(x) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned int* a, unsigned int x) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(x) : "memory");
}

template <class F>
__device__ __forceinline__ bool grid_sync_reduce(Ctrl* c, long long timeout_ns, int where, F&& on_last) {
  __shared__ int s_last, s_ok;
  __syncthreads();
  unsigned int g = 0;
  if (threadIdx.x == 0) {
    g = ld_relaxed_u32(&c->bar_gen);
    const unsigned int arrived = atom_add_acq_rel_u32(&c->bar_count, 1u);
    s_last = (arrived == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    // the sums of the next reduction go to the other set: clear it (every
    // CTA read it before arriving here)
    if (threadIdx.x < SC_STRIDE) c->acc_d[(where + 1) & 1][threadIdx.x] = 0.0;
    on_last(c->acc_d[where & 1]);
    __syncthreads();
    if (threadIdx.x == 0) {
      st_relaxed_u32(&c->bar_count, 0u);
      red_release_add_u32(&c->bar_gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile int* err = &c->err;
    unsigned long long t0 = globaltimer_ns();
    unsigned int ns = 32;
    while (ld_acquire_u32(&c->bar_gen) == g) {
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
  if (threadIdx.x == 0) s_ok = (*(volatile int*)&c->err == 0);
  __syncthreads();
  return s_ok != 0;
}

// Run by the last CTA: the K grid-wide sums into ctrl->red[0..K) as
// double-float values (read by every CTA after the barrier).
template <int K>
__device__ __forceinline__ void take_sums(Ctrl* c, const double* sums) {
  if (threadIdx.x < K) {
    const double d = __ldcg(sums + threadIdx.x);
    const float hi = (float)d;
    c->red[threadIdx.x] = make_float2(hi, (float)(d - (double)hi));
  }
  __syncthreads();
}

// After the barrier: the K reduced values, in every thread.
template <int K>
__device__ __forceinline__ void load_red(const Ctrl* c, df (&out)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 v = __ldcg(&c->red[k]);
    out[k] = {v.x, v.y};
  }
}

// --------------------------------------------------------------------------
// One tile of a pair pass
// --------------------------------------------------------------------------

// Rows of block I held by one lane: rows (a, a+1) packed in one f2x.
template <int DIM, int NC, int R>
struct Rows {
  f2x x[NC][DIM][R / 2];
  f2x acc[NC][DIM][R / 2];
};

#ifndef FD_MATVEC_RCP
#define FD_MATVEC_RCP 0
#endif
// 1/d^2 of an L^W product from the code itself (hardware reciprocal) instead
// of the table, on tiles that hold no code 0.
constexpr bool kMatvecRcp = FD_MATVEC_RCP != 0;

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The code in byte b of `codes` as a float plus 2^23 (exact for codes < 2^23).
__device__ __forceinline__ float code_plus_2p23(unsigned codes, unsigned b) {
  return __uint_as_float(__byte_perm(codes, 0x4B000000u, 0x7540u | b));
}

__device__ __forceinline__ float lut_at(const unsigned char* lut, unsigned off) {
  return *reinterpret_cast<const float*>(lut + off);
}

// Byte offset 256 * code + this lane's offset, for byte b of the code word.
__device__ __forceinline__ unsigned lut_off(unsigned codes, unsigned lane_off, unsigned b) {
  return __byte_perm(codes, lane_off, 0x5504u | (b << 4));
}

// Pairs this lane's rows with the G columns its group visits.  EDGE tiles
// (diagonal blocks, padding) may hold code 0 ("no pair"), whose stress term
// must vanish; elsewhere every code is a real distance.
template <int DIM, int MODE, int NC, int CODE, bool EDGE, int T = TILE>
__device__ __forceinline__ void tile_compute(const unsigned char* __restrict__ dt, const float* __restrict__ colv,
                                             const unsigned char* __restrict__ lut,
                                             Rows<DIM, NC, TileShape<DIM, MODE, T>::R>& rows, Vec<DIM> (&jout)[NC],
                                             float (&st)[NStress<MODE, NC>::v], int tid,
                                             int CA = T * DimP<DIM>::v /* floats between the candidate arrays */) {
  using TS = TileShape<DIM, MODE, T>;
  constexpr int R = TS::R, G = TS::G, CH = TS::CH;
  constexpr int DP = DimP<DIM>::v;
  constexpr bool NEED_K = (MODE != PM_MATVEC);
  constexpr bool NEED_W = (MODE == PM_MATVEC || MODE == PM_FORCES);
  const int q = tid & (G - 1), grp = tid / G;
  const unsigned off_k = 4u * (tid & 31), off_w = 128u + 4u * (tid & 31);
  // TINY keeps rsqrt finite for coincident points; it is below the FP32 resolution of r^2
  const f2x TINY2 = pk2(1e-30f, 1e-30f), NEG1 = pk2(-1.f, -1.f);
  constexpr int NS = NStress<MODE, NC>::v;
  float jacc[CH][NC][DIM];
  f2x stp[NS];
#pragma unroll
  for (int e = 0; e < NS; ++e) stp[e] = pk2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
#pragma unroll
    for (int h = 0; h < CH; ++h)
#pragma unroll
      for (int d = 0; d < DIM; ++d) jacc[h][c][d] = 0.f;
  }
#pragma unroll 1
  for (int t0 = 0; t0 < G; t0 += CH) {
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      const int jl = grp * G + ((q + t0 + h) & (G - 1));
      unsigned cw[(R + 3) / 4];
      float dv[(CODE == CODE_U8) ? 1 : R];
      if constexpr (CODE == CODE_U8) {
        const unsigned char* cp = dt + jl * T + R * q;
        if constexpr (R == 16) {
          const uint4 c = *reinterpret_cast<const uint4*>(cp);
          cw[0] = c.x;
          cw[1] = c.y;
          cw[2] = c.z;
          cw[3] = c.w;
        } else if constexpr (R == 8) {
          const uint2 c = *reinterpret_cast<const uint2*>(cp);
          cw[0] = c.x;
          cw[1] = c.y;
        } else {
          cw[0] = *reinterpret_cast<const unsigned*>(cp);
        }
      } else {
        const float4* cp = reinterpret_cast<const float4*>(dt) + (jl * T + R * q) / 4;
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
          const float4 v = cp[k];
          dv[4 * k] = v.x;
          dv[4 * k + 1] = v.y;
          dv[4 * k + 2] = v.z;
          dv[4 * k + 3] = v.w;
        }
      }
      f2x P[NC][DIM];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const Vec<DIM> pj = lds_v<DIM>(colv + c * CA, jl);
#pragma unroll
        for (int d = 0; d < DIM; ++d) P[c][d] = pk2(pj.c[d], pj.c[d]);
      }
      f2x J[NC][DIM];
#pragma unroll
      for (int a2 = 0; a2 < R / 2; ++a2) {
        f2x V = 0ull, W = 0ull, NEGM = NEG1;
        if constexpr (CODE == CODE_U8) {
          const unsigned c = cw[a2 >> 1];
          const unsigned b0 = (2u * a2) & 3u;
          if constexpr (NEED_K) V = pk2(lut_at(lut, lut_off(c, off_k, b0)), lut_at(lut, lut_off(c, off_k, b0 + 1)));
          if constexpr (MODE == PM_MATVEC && kMatvecRcp && !EDGE) {
            const f2x D = sub2(pk2(code_plus_2p23(c, b0), code_plus_2p23(c, b0 + 1)), pk2(8388608.f, 8388608.f));
            const f2x D2 = mul2(D, D);
            W = pk2(rcp_approx(lo2(D2)), rcp_approx(hi2(D2)));
          } else if constexpr (NEED_W) {
            W = pk2(lut_at(lut, lut_off(c, off_w, b0)), lut_at(lut, lut_off(c, off_w, b0 + 1)));
          }
        } else {
          // float tiles hold 1/d (0 for no pair)
          V = pk2(dv[2 * a2], dv[2 * a2 + 1]);
          W = mul2(V, V);
        }
        if constexpr ((EDGE || CODE != CODE_U8) &&
                      (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L || MODE == PM_ENUM))
          NEGM = pk2(lo2(V) > 0.f ? -1.f : 0.f, hi2(V) > 0.f ? -1.f : 0.f);
        if constexpr (MODE == PM_MATVEC) {
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            rows.acc[0][d][a2] = fma2(W, P[0][d], rows.acc[0][d][a2]);
            J[0][d] = (a2 == 0) ? mul2(W, rows.x[0][d][a2]) : fma2(W, rows.x[0][d][a2], J[0][d]);
          }
        } else if constexpr (MODE == PM_ENUM) {
          // candidate e: Delta = Delta_z + omega_e (Delta_z - Delta_x), omega_e = e / 2
          f2x DZ[DIM], DD[DIM];
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            DZ[d] = sub2(rows.x[0][d][a2], P[0][d]);
            DD[d] = sub2(DZ[d], sub2(rows.x[1][d][a2], P[1][d]));
          }
#pragma unroll
          for (int e = 0; e < NENUM; ++e) {
            const f2x OM = pk2(ENUM_STEP * e, ENUM_STEP * e);
            f2x R2 = TINY2;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              const f2x DE = fma2(OM, DD[d], DZ[d]);
              R2 = fma2(DE, DE, R2);
            }
            const f2x RS = pk2(rsqrt_approx(lo2(R2)), rsqrt_approx(hi2(R2)));
            const f2x TT = fma2(R2, mul2(RS, V), NEGM);  // r / d - 1
            stp[e] = fma2(TT, TT, stp[e]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            f2x DX[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) DX[d] = sub2(rows.x[c][d][a2], P[c][d]);
            f2x R2 = fma2(DX[0], DX[0], TINY2);
#pragma unroll
            for (int d = 1; d < DIM; ++d) R2 = fma2(DX[d], DX[d], R2);
            const f2x RS = pk2(rsqrt_approx(lo2(R2)), rsqrt_approx(hi2(R2)));
            f2x CO = mul2(RS, V);  // 1 / (d r)
            if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L) {
              const f2x TT = fma2(R2, CO, NEGM);  // r / d - 1
              stp[c] = fma2(TT, TT, stp[c]);
            }
            if constexpr (MODE == PM_FORCES) CO = sub2(CO, W);  // 1 / (d r) - 1 / d^2
            if constexpr (MODE != PM_STRESS) {
              if (MODE != PM_K2L || c == NC - 1) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                  rows.acc[c][d][a2] = fma2(CO, DX[d], rows.acc[c][d][a2]);
                  J[c][d] = (a2 == 0) ? mul2(CO, DX[d]) : fma2(CO, DX[d], J[c][d]);
                }
              }
            }
          }
        }
      }
      if constexpr (MODE != PM_STRESS && MODE != PM_ENUM) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            if (MODE == PM_K2L && c != NC - 1) continue;
            jacc[h][c][d] += lo2(J[c][d]);
            jacc[h][c][d] += hi2(J[c][d]);
            if constexpr (CH < G) jacc[h][c][d] = __shfl_sync(0xffffffffu, jacc[h][c][d], (q + CH) & (G - 1), G);
          }
      }
    }
  }
  // chain h of lane q now holds column (q + h) mod G of the group: gather column q
#pragma unroll
  for (int e = 0; e < NS; ++e) st[e] = lo2(stp[e]) + hi2(stp[e]);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if constexpr (MODE == PM_K2L) {
      if (c != NC - 1) {
        jout[c] = vzero<DIM>();
        continue;
      }
    }
    if constexpr (MODE != PM_STRESS && MODE != PM_ENUM) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        float s = jacc[0][c][d];
#pragma unroll
        for (int h = 1; h < CH; ++h) s += __shfl_sync(0xffffffffu, jacc[h][c][d], (q - h) & (G - 1), G);
        jout[c].c[d] = s;
      }
    }
  }
}

// Forms element t of block blk of the pass's vectors, in place in the raw
// arrays (candidate c goes to array c's slot): raw is the block's part of
// array 0, A the floats between arrays, sc the block's scalars (SK_CGU).
template <int DIM, int NC>
__device__ __forceinline__ void form_inplace(const PassSrc& s, float* raw, int blk, int t, int A, const float* sc) {
  constexpr int DP = DimP<DIM>::v;
  const int kind = s.kind;
  if (kind == SK_CGU) {
    const Vec<DIM> r = lds_v<DIM>(raw, t);
    const Vec<DIM> w = lds_v<DIM>(raw + A, t);
    const Vec<DIM> sp = lds_v<DIM>(raw + 2 * A, t);
    const float is = sc[t];
    Vec<DIM> u;
#pragma unroll
    for (int d = 0; d < DIM; ++d) u.c[d] = cg_u(r.c[d], w.c[d], sp.c[d], is, s.alpha[d], s.beta[d]);
    sts_v<DIM>(raw, t, u);
  } else if (kind == SK_K2 || kind == SK_SEL || kind == SK_ZX) {
    const Vec<DIM> zw = lds_v<DIM>(raw, t);
    Vec<DIM> z;
#pragma unroll
    for (int d = 0; d < DIM; ++d) z.c[d] = zw.c[d] - s.z0[d];
    // omega_i of vertex blk * TILE + t (the padding's factors are 0)
    const float mi = s.oms ? __ldg(s.oms + (size_t)blk * TILE + t) : 1.f;
    const float om = s.oms ? s.om * mi : s.om;
    if (kind == SK_K2 && NC == 2) {
      const Vec<DIM> x = lds_v<DIM>(raw + A, t);
      Vec<DIM> xt;
#pragma unroll
      for (int d = 0; d < DIM; ++d) xt.c[d] = sor_xt(z.c[d], x.c[d], om);
      sts_v<DIM>(raw + A, t, xt);
    }
    if (kind == SK_ZX && s.oms) {
      // the enumeration pass forms z + omega_e (z - x) pairwise; with
      // per-vertex factors its second vector is z - m_i (z - x)
      const Vec<DIM> x = lds_v<DIM>(raw + A, t);
      Vec<DIM> xm;
#pragma unroll
      for (int d = 0; d < DIM; ++d) xm.c[d] = fmaf(-mi, z.c[d] - x.c[d], z.c[d]);
      sts_v<DIM>(raw + A, t, xm);
    }
    if (kind == SK_SEL && s.sel) {
      const Vec<DIM> x = lds_v<DIM>(raw + A, t);
#pragma unroll
      for (int d = 0; d < DIM; ++d) z.c[d] = sor_xt(z.c[d], x.c[d], om);
    }
    sts_v<DIM>(raw, t, z);
  }
}

// Thread 0 of a CTA: bulk copies (TMA) of a step's c tiles (consecutive in
// the strip, so their codes are one copy) and of the raw source arrays of
// their column blocks (one copy per array when the blocks are consecutive),
// and, at a task's first step, of block I; all complete on the stage's
// mbarrier.
template <int DIM, int CODE, int TPS>
__device__ __forceinline__ void issue_tile(const PassArgs& p, const PassSrc& src, unsigned char* smem, int tile, int I,
                                        int J, int c, bool first, int s) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  constexpr unsigned TBYTES = L::DBUF;
  constexpr int tps = TPS;
  const int kind = src.kind;
  const int NA = src_arrays(kind);
  const unsigned RB = raw_bytes<DIM>(kind);
  const int sb = p.stage_base;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC) + s;
  fence_proxy_async();  // this CTA's generic accesses to the stage come before the copy overwrites it
  mbar_expect_tx(mbar, c * (TBYTES + RB) + (first ? RB : 0));
  bulk_g2s(smem + L::off_d(sb, s, tps), reinterpret_cast<const unsigned char*>(p.D) + (size_t)tile * TBYTES, c * TBYTES,
           mbar);
  // column blocks J, J + 1 (mod nb): one run of c blocks, or two runs at the wrap
  float* rawj = reinterpret_cast<float*>(smem + L::off_rawj(sb, s, tps));
  const int run0 = (J + c <= p.nb) ? c : 1;
  for (int a = 0; a < NA; ++a) {
    const bool scalar = (kind == SK_CGU && a == 3);
    const unsigned ab = scalar ? TILE * 4 : TILE * DP * 4;  // bytes of one block
    const int stride = scalar ? TILE : TILE * DP;           // floats of one block
    float* dst = scalar ? rawj + 3 * tps * TILE * DP : rawj + a * tps * TILE * DP;
    bulk_g2s(dst, src.a[a] + (size_t)J * stride, run0 * ab, mbar);
    if (run0 < c) bulk_g2s(dst + stride, src.a[a], ab, mbar);  // block 0 after block nb - 1
  }
  if (first) {
    float* rawi = reinterpret_cast<float*>(smem + L::off_rawi(sb, s, tps));
    for (int a = 0; a < NA; ++a) {
      const bool scalar = (kind == SK_CGU && a == 3);
      const unsigned ab = scalar ? TILE * 4 : TILE * DP * 4;
      const int stride = scalar ? TILE : TILE * DP;
      bulk_g2s(rawi + a * TILE * DP, src.a[a] + (size_t)I * stride, ab, mbar);
    }
  }
}

// Iterations between the all-pairs passes that recompute L^W x0 at the start
// of an H step (in between it comes from the previous step's vectors).
constexpr int LWX_REFRESH = 16;

// Whether a step's copies are issued by four warps (issue_step_part) or all
// by thread 0 (issue_tile).  Measured at n = 200,000: with two tiles per
// stage the split takes 7-10 % off an L^W pass in 2-D; with one tile per
// stage (3-D, before it took two-tile stages) it made the pass 2 % slower.
template <int TPS>
constexpr bool kSplitIssue = (TPS == 2);

// One step's copies, as the thread that prepares them describes them to the
// warps that issue them (two alternating slots in shared memory).
struct IssueDesc {
  int tile, I, J;
  int flags;  // c | first << 8 | stage << 16 | valid << 24
  __device__ __forceinline__ int c() const { return flags & 0xff; }
  __device__ __forceinline__ bool first() const { return ((flags >> 8) & 1) != 0; }
  __device__ __forceinline__ int stage() const { return (flags >> 16) & 0xff; }
  __device__ __forceinline__ bool valid() const { return (flags >> 24) != 0; }
};

// The copy issue of one step spread over the CTA's four warps: lane 0 of
// warp 0 arms the stage's mbarrier with the step's bytes and copies the
// codes; lane 0 of warp (a + 1) mod 4 copies raw array a (its column blocks
// and, at a task's first step, block I).  A copy may complete before the
// mbarrier is armed: the transaction count goes negative until the armed
// arrival, and the phase cannot complete without that arrival.
template <int DIM, int CODE, int TPS>
__device__ __forceinline__ void issue_step_part(const PassArgs& p, const PassSrc& src, unsigned char* smem,
                                                const IssueDesc& d, int warp) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  constexpr unsigned TBYTES = L::DBUF;
  constexpr int tps = TPS;
  const int kind = src.kind;
  const int NA = src_arrays(kind);
  const int c = d.c(), s = d.stage(), J = d.J;
  const bool first = d.first();
  const int sb = p.stage_base;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC) + s;
  fence_proxy_async();  // this CTA's generic accesses to the stage come before the copy overwrites it
  if (warp == 0) {
    const unsigned RB = raw_bytes<DIM>(kind);
    mbar_expect_tx(mbar, c * (TBYTES + RB) + (first ? RB : 0));
    bulk_g2s(smem + L::off_d(sb, s, tps), reinterpret_cast<const unsigned char*>(p.D) + (size_t)d.tile * TBYTES,
             c * TBYTES, mbar);
  }
  float* rawj = reinterpret_cast<float*>(smem + L::off_rawj(sb, s, tps));
  float* rawi = reinterpret_cast<float*>(smem + L::off_rawi(sb, s, tps));
  const int run0 = (J + c <= p.nb) ? c : 1;
  for (int a = 0; a < NA; ++a) {
    if (((a + 1) & 3) != warp) continue;
    const bool scalar = (kind == SK_CGU && a == 3);
    const unsigned ab = scalar ? TILE * 4 : TILE * DP * 4;  // bytes of one block
    const int stride = scalar ? TILE : TILE * DP;           // floats of one block
    float* dst = scalar ? rawj + 3 * tps * TILE * DP : rawj + a * tps * TILE * DP;
    bulk_g2s(dst, src.a[a] + (size_t)J * stride, run0 * ab, mbar);
    if (run0 < c) bulk_g2s(dst + stride, src.a[a], ab, mbar);  // block 0 after block nb - 1
    if (first) bulk_g2s(rawi + a * TILE * DP, src.a[a] + (size_t)d.I * stride, ab, mbar);
  }
}

// The steps of one CTA in visiting order: its tasks m = 0..M-1 and, inside a
// task, runs of c = tps consecutive tiles (fewer at the task's end) in strip
// order; both reversed when `rev` (a step's tiles are k .. k + c - 1 either way).
template <int TPS>
struct TileIt {
  int m, k, c, M;
  bool rev, valid;
  TaskDesc td;
  __device__ __forceinline__ void set_from_hi(int hi) {  // reversed: the step ending at tile hi
    k = max(td.k0, hi - TPS + 1);
    c = hi - k + 1;
  }
  __device__ __forceinline__ void load(const PassArgs& g) {
    const int mm = rev ? (M - 1 - m) : m;
    td = (mm < MAX_CTA_TASKS) ? g.tasks_s[mm] : g.tasks_g[mm];
    if (rev) {
      set_from_hi(td.k1 - 1);
    } else {
      k = td.k0;
      c = min(TPS, td.k1 - td.k0);
    }
  }
  __device__ __forceinline__ void begin(const PassArgs& g, bool r) {
    rev = r;
    M = g.ntasks;
    m = 0;
    valid = M > 0;
    if (valid) load(g);
  }
  __device__ __forceinline__ bool first() const { return rev ? (k + c == td.k1) : (k == td.k0); }
  __device__ __forceinline__ bool last() const { return rev ? (k == td.k0) : (k + c == td.k1); }
  __device__ __forceinline__ void next(const PassArgs& g) {
    if (!last()) {
      if (rev) {
        set_from_hi(k - 1);
      } else {
        k += c;
        c = min(TPS, td.k1 - k);
      }
      return;
    }
    if (++m >= M) {
      valid = false;
      return;
    }
    load(g);
  }
  // column block of the step's first tile (k < nb, so one subtraction wraps it)
  __device__ __forceinline__ int J(int nb) const {
    const int j = td.I + k;
    return (j >= nb) ? j - nb : j;
  }
  __device__ __forceinline__ int tile() const { return td.tile0 + (k - td.k0); }
};

// A pass's parameters, kept in shared memory (read where they are used, so
// that the tile loop keeps its registers), and the copy issuer's iterator.
struct PassCtl {
  PassSrc src;
  PassArgs a;
  TileIt<1> is;  // the step after the one in desc (thread 0 only; TileIt<2> has the same layout)
  int s_is;      // its stage
  IssueDesc desc[2];  // the step whose copies the loop's step t issues: desc[t & 1]
};
static_assert(sizeof(TileIt<1>) == sizeof(TileIt<2>), "step iterators share the PassCtl slot");
static_assert(sizeof(PassCtl) <= SmemLayout<1, CODE_U8>::OFF_RUN - SmemLayout<1, CODE_U8>::OFF_CTL,
              "PassCtl must fit its shared-memory slot");

// Scalars of the Algorithm 2 loop (shared memory, written by thread 0).
struct RunState {
  double f_cur, f_new, crit, passes_mv, passes_st, f_enum0, passes_en;
  int cg_total, cg_maxed, cg_stalled, n_acc, it_outer, it;
  int accept, bsel, stop, all_conv, cg_done, cg_last;
  int conv[3];
  float z0[3], om_prev;
  float alpha[3], beta[3], gam[3], rz[3], bb[3];
};
static_assert(sizeof(RunState) <= SmemLayout<1, CODE_U8>::OFF_PARAMS - SmemLayout<1, CODE_U8>::OFF_RUN,
              "RunState must fit its shared-memory slot");
static_assert(sizeof(KParams) <= SmemLayout<1, CODE_U8>::OFF_TASKS - SmemLayout<1, CODE_U8>::OFF_PARAMS,
              "KParams must fit its shared-memory slot");

// --------------------------------------------------------------------------
// A full pair pass: CTA b takes tasks b, b + G, b + 2G, ... (G = grid size);
// no global synchronisation inside the pass.  Row and column sums go to
// acc + c * n_pad * DP (candidate c); stress to the CTA's slot.  Out of line,
// so that the tile loop has the registers to itself.
// --------------------------------------------------------------------------

#ifndef FD_PASS_ATTR
#define FD_PASS_ATTR __noinline__
#endif
template <int DIM, int MODE, int NC, int CODE, int TPS>
__device__ FD_PASS_ATTR bool pair_pass_impl(PairState* ps_io, double* acc) {
  // the dynamic shared memory itself (not a pointer argument), so that every
  // access compiles to a shared-memory instruction with a constant base
  extern __shared__ __align__(256) unsigned char smem[];
  using L = SmemLayout<DIM, CODE>;
  using TS = TileShape<DIM, MODE>;
  constexpr int R = TS::R, G = TS::G;
  constexpr int DP = DimP<DIM>::v;
  PassCtl* ctl = reinterpret_cast<PassCtl*>(smem + L::OFF_CTL);
  const PassArgs& p = ctl->a;
  const PassArgs& g = ctl->a;
  const PassSrc& src = ctl->src;
  PairState ps = *ps_io;
  const int tid = threadIdx.x, nbuf = p.nbuf;
  const size_t vs = (size_t)g.n_pad * DP;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
  float2* red64 = reinterpret_cast<float2*>(smem + L::OFF_RED64);
  const unsigned char* lut = smem + L::OFF_LUT;
  const int sb = p.stage_base;
  constexpr int NS = NStress<MODE, NC>::v;
  float ssum[NS], scomp[NS];
#pragma unroll
  for (int c = 0; c < NS; ++c) ssum[c] = scomp[c] = 0.f;
  // vectors written before the last grid barrier are read below by bulk copies
  if (tid == 0) fence_proxy_async_global();
  const bool rev = (ps.pass & 1) != 0;
  TileIt<TPS> it;  // computed step
  it.begin(g, rev);
  int s_it = 0;  // its stage
  TileIt<TPS>& ctl_is = *reinterpret_cast<TileIt<TPS>*>(&ctl->is);
  // describes the step at ctl_is (its stage ctl->s_is) into desc[slot] and moves past it
  auto prepare = [&](int slot) {
    TileIt<TPS> is = ctl_is;
    IssueDesc d;
    d.tile = is.valid ? is.tile() : 0;
    d.I = is.valid ? is.td.I : 0;
    d.J = is.valid ? is.J(g.nb) : 0;
    d.flags = is.valid ? (is.c | (is.first() ? 1 << 8 : 0) | (ctl->s_is << 16) | (1 << 24)) : 0;
    ctl->desc[slot] = d;
    if (is.valid) {
      is.next(g);
      ctl_is = is;
      ctl->s_is = (ctl->s_is + 1 == nbuf) ? 0 : ctl->s_is + 1;
    }
  };
  if (tid == 0) {
    TileIt<TPS> is = it;
    int s_is = 0;
    for (int k = 0; k < nbuf - 1 && is.valid; ++k) {
      issue_tile<DIM, CODE, TPS>(p, src, smem, is.tile(), is.td.I, is.J(g.nb), is.c, is.first(), s_is);
      is.next(g);
      s_is = (s_is + 1 == nbuf) ? 0 : s_is + 1;
    }
    ctl_is = is;
    ctl->s_is = s_is;
    if constexpr (kSplitIssue<TPS>) prepare(0);
  }
  int t_step = 0;
  Rows<DIM, NC, R> rows;
  constexpr int tps = TPS;
  constexpr int astr = TPS * TILE * DP;  // floats between the raw arrays of the column blocks
  while (it.valid) {
    const int I = it.td.I, J0 = it.J(g.nb), nc = it.c;
    const bool first = it.first(), last = it.last();
    const unsigned ph = (ps.parity >> s_it) & 1u;
    if (!mbar_wait(mbar + s_it, ph, p.timeout_ns)) {
      set_error(p.ctrl, E_TIMEOUT);
      // let this CTA's own copies land (bounded) before leaving
      for (int k = 0; k < nbuf; ++k) mbar_wait(mbar + k, (ps.parity >> k) & 1u, p.timeout_ns);
      *ps_io = ps;
      return false;
    }
    ps.parity ^= (1u << s_it);
    float* rawj = reinterpret_cast<float*>(smem + L::off_rawj(sb, s_it, tps));
    float* rawi = reinterpret_cast<float*>(smem + L::off_rawi(sb, s_it, tps));
    form_inplace<DIM, NC>(src, rawj, J0, tid, astr, rawj + 3 * astr);
    if constexpr (TPS == 2) {
      if (nc == 2)
        form_inplace<DIM, NC>(src, rawj + TILE * DP, (J0 + 1 == g.nb) ? 0 : J0 + 1, tid, astr,
                              rawj + 3 * astr + TILE);
    }
    if (first) form_inplace<DIM, NC>(src, rawi, I, tid, TILE * DP, rawi + 3 * TILE * DP);
    __syncthreads();  // formed vectors visible; every thread is done with the stage of the previous step
    if constexpr (kSplitIssue<TPS>) {
      // the copies of the step nbuf - 1 ahead, lane 0 of each warp a part
      const IssueDesc& d = ctl->desc[t_step & 1];
      if ((tid & 31) == 0 && d.valid()) issue_step_part<DIM, CODE, TPS>(p, src, smem, d, tid >> 5);
      if (tid == 0) prepare((t_step + 1) & 1);
      ++t_step;
    } else if (tid == 0 && ctl_is.valid) {
      TileIt<TPS> is = ctl_is;
      issue_tile<DIM, CODE, TPS>(p, src, smem, is.tile(), is.td.I, is.J(g.nb), is.c, is.first(), ctl->s_is);
      is.next(g);
      ctl_is = is;
      ctl->s_is = (ctl->s_is + 1 == nbuf) ? 0 : ctl->s_is + 1;
    }
    const int q = tid & (G - 1);
    if (first) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int a2 = 0; a2 < R / 2; ++a2) {
          const Vec<DIM> x0 = lds_v<DIM>(rawi + c * TILE * DP, R * q + 2 * a2);
          const Vec<DIM> x1 = lds_v<DIM>(rawi + c * TILE * DP, R * q + 2 * a2 + 1);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            rows.x[c][d][a2] = pk2(x0.c[d], x1.c[d]);
            rows.acc[c][d][a2] = pk2(0.f, 0.f);
          }
        }
    }
    // the step's tiles: u = 0, and u = 1 when the step holds two
    auto do_tile = [&](int u) {
      const int Ju = (J0 + u >= g.nb) ? J0 + u - g.nb : J0 + u;
      Vec<DIM> jout[NC];
      float st[NS];
      const unsigned char* dt = smem + L::off_d(sb, s_it, tps) + u * L::DBUF;
      const float* colv = rawj + u * TILE * DP;
      const bool edge = (it.k + u == 0) || (g.n < g.n_pad && (I == g.nb - 1 || Ju == g.nb - 1));
      if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L || MODE == PM_ENUM ||
                    (MODE == PM_MATVEC && kMatvecRcp)) {
        if (edge) tile_compute<DIM, MODE, NC, CODE, true>(dt, colv, lut, rows, jout, st, tid, astr);
        else tile_compute<DIM, MODE, NC, CODE, false>(dt, colv, lut, rows, jout, st, tid, astr);
      } else {
        tile_compute<DIM, MODE, NC, CODE, false>(dt, colv, lut, rows, jout, st, tid, astr);
      }
      if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L || MODE == PM_ENUM) {
#pragma unroll
        for (int c = 0; c < NS; ++c) kahan_add(ssum[c], scomp[c], st[c]);
      }
      if constexpr (MODE != PM_STRESS && MODE != PM_ENUM) {
        // column sums: thread t holds column t of block Ju
        const int j = Ju * TILE + tid;
        if (j < g.n) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (MODE == PM_K2L && c != NC - 1) continue;
            Vec<DIM> v = jout[c];
            if constexpr (MODE != PM_MATVEC) {
#pragma unroll
              for (int d = 0; d < DIM; ++d) v.c[d] = -v.c[d];
            }
            atomic_addv<DIM>(acc + c * vs, j, v);
          }
        }
      }
    };
    do_tile(0);
    if constexpr (TPS == 2) {
      if (nc == 2) do_tile(1);
    }
    if constexpr (MODE != PM_STRESS && MODE != PM_ENUM) {
      if (last) {
        // row sums of the task: the R groups' partials meet in the stage's code buffer
        float* red = reinterpret_cast<float*>(smem + L::off_d(sb, s_it, tps));  // [NC][R groups][TILE][DP]
        const int grp = tid / G;
        __syncthreads();  // every warp is done with the codes
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int a2 = 0; a2 < R / 2; ++a2) {
            if (MODE == PM_K2L && c != NC - 1) continue;
            Vec<DIM> v0, v1;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              v0.c[d] = lo2(rows.acc[c][d][a2]);
              v1.c[d] = hi2(rows.acc[c][d][a2]);
            }
            float* base = red + ((size_t)(c * R + grp) * TILE) * DP;
            sts_v<DIM>(base, R * q + 2 * a2, v0);
            sts_v<DIM>(base, R * q + 2 * a2 + 1, v1);
          }
        __syncthreads();
        const int i = I * TILE + tid;
        if (i < g.n) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (MODE == PM_K2L && c != NC - 1) continue;
            Vec<DIM> s = lds_v<DIM>(red + ((size_t)(c * R) * TILE) * DP, tid);
#pragma unroll
            for (int gg = 1; gg < R; ++gg) {
              const Vec<DIM> v = lds_v<DIM>(red + ((size_t)(c * R + gg) * TILE) * DP, tid);
#pragma unroll
              for (int d = 0; d < DIM; ++d) s.c[d] += v.c[d];
            }
            atomic_addv<DIM>(acc + c * vs, i, s);
          }
        }
      }
    }
    it.next(g);
    s_it = (s_it + 1 == nbuf) ? 0 : s_it + 1;
  }
  // stress of this CTA's pairs (per candidate), double-float slots per CTA
  if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L || MODE == PM_ENUM) {
    df v[NS];
#pragma unroll
    for (int c = 0; c < NS; ++c) v[c] = df_add(df_of(ssum[c]), df_of(-scomp[c]));
    cta_sum_multi<NS>(v, red64);
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < NS; ++c) atomicAdd(p.rsum + c, df_to_double(v[c]));
    }
  }
  ps.pass += 1;
  *ps_io = ps;
  return true;
}

template <int DIM, int MODE, int NC, int CODE, int TPS>
__device__ __forceinline__ bool pair_pass(const KParams& p, unsigned char* smem, PairState& ps, const PassSrc& src,
                                          double* acc, double* rsum = nullptr) {
  using L = SmemLayout<DIM, CODE>;
  PassCtl* ctl = reinterpret_cast<PassCtl*>(smem + L::OFF_CTL);
  if (threadIdx.x == 0) {
    ctl->src = src;
    PassArgs& a = ctl->a;
    a.D = p.D;
    const int t0 = p.g.cta_task_ptr[blockIdx.x];
    a.tasks_g = p.g.tasks + t0;
    a.tasks_s = reinterpret_cast<const TaskDesc*>(smem + L::OFF_TASKS);
    a.ctrl = p.ctrl;
    a.rsum = rsum;
    a.timeout_ns = p.timeout_ns;
    a.n = p.g.n;
    a.n_pad = p.g.n_pad;
    a.nb = p.g.nb;
    a.ntasks = p.g.cta_task_ptr[blockIdx.x + 1] - t0;
    a.nbuf = p.nbuf;
    a.stage_base = L::stage_base(CODE == CODE_U8 ? p.lut_rows * LUT_ROW : 0);
    a.tps = p.tps;
  }
  __syncthreads();
  return pair_pass_impl<DIM, MODE, NC, CODE, TPS>(&ps, acc);
}

// --------------------------------------------------------------------------
// Vertex phase: one thread per vertex (CTA b takes vertex blocks b, b + G,
// ...); fn(i, v) adds the vertex's K scalars to v, which the CTA sums and
// adds to the grid-wide sums rsum (FP64 atomics).
// --------------------------------------------------------------------------
template <int K, class F>
__device__ __forceinline__ void vertex_phase(const KParams& p, float2* red64, double* rsum, F&& fn) {
  constexpr int K1 = (K > 0) ? K : 1;
  df v[K1];
#pragma unroll
  for (int k = 0; k < K1; ++k) v[k] = df_of(0.f);
  for (int blk = blockIdx.x; blk < p.g.nb; blk += gridDim.x) fn(blk * TILE + (int)threadIdx.x, v);
  if constexpr (K > 0) {
    cta_sum_multi<K>(v, red64);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) atomicAdd(rsum + k, df_to_double(v[k]));
    }
  }
}

// --------------------------------------------------------------------------
// Direct solver: z = A'^-1 r with the dense inverse of the shifted L^W
// (L^W + sigma/n 1 1^T, inverted once before the launch).  The inverse is
// streamed once from HBM with 16-byte loads; a CTA takes 8 rows and half of
// the columns at a time (2 rows per warp, each lane 4 consecutive columns),
// r goes through shared memory in chunks of DCH vertices, one coordinate per
// array (so that a lane's 4 vertices are one 16-byte read), double-buffered
// through registers.  Every partial sum has one fixed order and each row gets
// two: the result does not depend on the grid.  z must be zero on entry.
// --------------------------------------------------------------------------
constexpr int DCH = 1024;  // vertices per staged chunk of r

template <int DIM>
__device__ __noinline__ void dense_apply(const KParams& p, float* buf, const float* __restrict__ r,
                                            float* __restrict__ z) {
  constexpr int DP = DimP<DIM>::v;
  constexpr int PT = DCH * DP / 4 / CTA;  // float4 of a chunk per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int np = p.g.n_pad;  // a multiple of TILE
  const int nch = (np + DCH - 1) / DCH;
  float4 pre[PT];
  auto fetch = [&](int ch) {
    const float4* src = reinterpret_cast<const float4*>(r + (size_t)ch * DCH * DP);
    const int lim = min(DCH, np - ch * DCH) * DP / 4;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int idx = threadIdx.x + q * CTA;
      pre[q] = (idx < lim) ? __ldcg(src + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto put = [&](float* b) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int idx = threadIdx.x + q * CTA;
      const float4 v = pre[q];
      if constexpr (DP == 1) {
        reinterpret_cast<float4*>(b)[idx] = v;
      } else if constexpr (DP == 2) {
        reinterpret_cast<float2*>(b)[idx] = make_float2(v.x, v.z);
        reinterpret_cast<float2*>(b + DCH)[idx] = make_float2(v.y, v.w);
      } else {
        b[idx] = v.x;
        b[DCH + idx] = v.y;
        b[2 * DCH + idx] = v.z;
      }
    }
  };
  // Work items: (row group, column half).  Halving the columns doubles the
  // items, so that the last round over the grid is nearly full; each row
  // receives its two partial sums by atomic adds into z, which is zero on
  // entry (two adds into zero give the same result in either order).
  const int half = (nch + 1) / 2;
  for (int it = blockIdx.x; it < np / 4; it += gridDim.x) {
    const int gi = it >> 1, h = it & 1;
    const int ch0 = h * half, ch1 = min(nch, ch0 + half);
    if (ch0 >= ch1) continue;  // one chunk only: the second half is empty (uniform over the CTA)
    const int i0 = gi * 8 + warp * 2;
    const float* a0 = p.ainv + (size_t)i0 * np;
    const float* a1 = a0 + np;
    float s0[DIM], s1[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) s0[d] = s1[d] = 0.f;
    fetch(ch0);
    put(buf);
    __syncthreads();
    for (int ch = ch0; ch < ch1; ++ch) {
      if (ch + 1 < ch1) fetch(ch + 1);
      const float* rb = buf + ((ch - ch0) & 1) * DIM * DCH;
      const int c0 = ch * DCH, len = min(DCH, np - c0);
#pragma unroll 4
      for (int c = lane * 4; c < len; c += 128) {
        const float4 u0 = __ldcs(reinterpret_cast<const float4*>(a0 + c0 + c));
        const float4 u1 = __ldcs(reinterpret_cast<const float4*>(a1 + c0 + c));
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float4 v = *reinterpret_cast<const float4*>(rb + d * DCH + c);
          s0[d] = fmaf(u0.x, v.x, fmaf(u0.y, v.y, fmaf(u0.z, v.z, fmaf(u0.w, v.w, s0[d]))));
          s1[d] = fmaf(u1.x, v.x, fmaf(u1.y, v.y, fmaf(u1.z, v.z, fmaf(u1.w, v.w, s1[d]))));
        }
      }
      if (ch + 1 < ch1) put(buf + ((ch + 1 - ch0) & 1) * DIM * DCH);
      __syncthreads();
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0[d] += __shfl_xor_sync(0xffffffffu, s0[d], o);
        s1[d] += __shfl_xor_sync(0xffffffffu, s1[d], o);
      }
    if (lane == 0) {
      Vec<DIM> v0, v1;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        v0.c[d] = s0[d];
        v1.c[d] = s1[d];
      }
      atomic_addv<DIM>(z, i0, v0);
      atomic_addv<DIM>(z, i0 + 1, v1);
    }
  }
}

// Reads and clears accumulator entry i.
template <int DIM>
__device__ __forceinline__ Vec<DIM> take_acc(float* a, int i) {
  const Vec<DIM> v = ldv<DIM>(a, i);
  stv<DIM>(a, i, vzero<DIM>());
  return v;
}
template <int DIM>
__device__ __forceinline__ Vec<DIM> take_acc(double* a, int i) {
  constexpr int DP = DimP<DIM>::v;
  Vec<DIM> v;
  if constexpr (DIM == 1) {
    v.c[0] = (float)__ldcg(a + i);
    __stcg(a + i, 0.0);
  } else {
    // DP = 2 or 4 doubles per vertex: 16-byte aligned pairs
    const double2* q = reinterpret_cast<const double2*>(a + (size_t)DP * i);
    const double2 t0 = __ldcg(q);
    v.c[0] = (float)t0.x;
    v.c[1] = (float)t0.y;
    if constexpr (DIM == 3) v.c[2] = (float)__ldcg(q + 1).x;
    double2* w = reinterpret_cast<double2*>(a + (size_t)DP * i);
    __stcg(w, make_double2(0.0, 0.0));
    if constexpr (DIM == 3) __stcg(w + 1, make_double2(0.0, 0.0));
  }
  return v;
}

__device__ __forceinline__ PassSrc direct_src(const float* a, int kind = SK_DIRECT) {
  PassSrc s;
  s.kind = kind;
  s.a[0] = a;
  s.a[1] = s.a[2] = s.a[3] = nullptr;
#pragma unroll
  for (int d = 0; d < 3; ++d) s.alpha[d] = s.beta[d] = s.z0[d] = 0.f;
  s.om = 0.f;
  s.sel = 0;
  s.oms = nullptr;
  return s;
}

// --------------------------------------------------------------------------
// The kernel
// --------------------------------------------------------------------------

// WITH_ENUM: the variant that also runs the enumerating strategy (its pass is
// kept out of the other variant, whose passes then keep their registers).
// TPS: tiles per pipeline stage (a kernel of its own, so that every kernel
// calls one variant of each pass).
template <int DIM, int CODE, bool WITH_ENUM, int TPS = 1>
__global__ void __launch_bounds__(CTA, 2) fd_main_kernel(KParams p_in) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  extern __shared__ __align__(256) unsigned char smem[];
  // The parameters are read from a shared-memory copy: values that the
  // compiler cannot keep in registers across the out-of-line passes.
  {
    static_assert(sizeof(KParams) % 8 == 0, "KParams copy granularity");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&p_in);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(smem + L::OFF_PARAMS);
    for (int k = threadIdx.x; k < (int)(sizeof(KParams) / 8); k += CTA) dst[k] = src[k];
    __syncthreads();
  }
  const KParams& p = *reinterpret_cast<const KParams*>(smem + L::OFF_PARAMS);
  const Geometry& g = p.g;
  {
    const int t0 = p_in.g.cta_task_ptr[blockIdx.x], t1 = p_in.g.cta_task_ptr[blockIdx.x + 1];
    TaskDesc* ts = reinterpret_cast<TaskDesc*>(smem + L::OFF_TASKS);
    for (int k = threadIdx.x; k < min(t1 - t0, MAX_CTA_TASKS); k += CTA) ts[k] = p_in.g.tasks[t0 + k];
    __syncthreads();
  }
  // Everything below is re-derived from the shared-memory copy where it is
  // used, so that nothing but loop counters stays live across a pass.
#define n (p.g.n)
#define nb (p.g.nb)
#define tid ((int)threadIdx.x)
#define vs ((size_t)p.g.n_pad * DP)
#define acc0 (p.acc)           /* RHS of candidate 0, forces */
#define acc1 (p.acc + vs)      /* RHS of candidate 1 */
#define acc2 (p.acc + 2 * vs)  /* L^W products */
#define red64 (reinterpret_cast<float2*>(smem + L::OFF_RED64))
#define ctrl (p.ctrl)

  // --- set-up: mbarriers and the replicated lookup table
  {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
    if (tid == 0) {
      for (int k = 0; k < p.nbuf; ++k) mbar_init(&mbar[k], 1);
      fence_mbar_init();
    }
    if constexpr (CODE == CODE_U8) {
      uint4* dst = reinterpret_cast<uint4*>(smem + L::OFF_LUT);
      const uint4* srcl = reinterpret_cast<const uint4*>(p.lut);
      for (int k = tid; k < p.lut_rows * (LUT_ROW / 16); k += CTA) dst[k] = srcl[k];
    }
    __syncthreads();
  }
  PairState ps;
  ps.parity = 0u;
  ps.pass = 0;
  int nbar = 0;
  // start of the launch for the per-iteration times (read by CTA 0, thread 0 only)
  const unsigned long long t_launch = (blockIdx.x == 0 && tid == 0) ? globaltimer_ns() : 0ull;
  if (p.timeline && blockIdx.x == 0 && tid == 0) ctrl->t_start = globaltimer_ns();
  auto mark = [&](int tag) {
    if (p.timeline && blockIdx.x == 0 && tid == 0 && ctrl->timeline_n < p.timeline_cap) {
      const int q = ctrl->timeline_n++;
      p.timeline[2 * q] = (double)tag;
      p.timeline[2 * q + 1] = (double)(globaltimer_ns() - ctrl->t_start);
    }
  };
  auto no_reduction = [](const double*) {};
  // grid barrier; the last CTA to arrive runs `red` on the grid-wide sums first
#define FD_SYNC_RED(tag, red)                                                   \
  do {                                                                          \
    if (!grid_sync_reduce(ctrl, p.bar_timeout_ns, ++nbar, red)) return;         \
    mark(tag);                                                                  \
  } while (0)
#define FD_SYNC(tag) FD_SYNC_RED(tag, no_reduction)
  // the grid-wide sums the next reduction barrier (index nbar + 1) collects
#define RSUM (ctrl->acc_d[(nbar + 1) & 1])
  auto red_stress = [&](int nc) {
    return [&, nc](const double* sums) {
      if (nc == 2) take_sums<2>(ctrl, sums);
      else take_sums<1>(ctrl, sums);
    };
  };

  // --- pack the caller layout into the padded internal array, check it; clear the accumulators
  for (int R = blockIdx.x; R < nb; R += gridDim.x) {
    const int i = R * TILE + tid;
    Vec<DIM> v;
    bool bad = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      float x = (i < n) ? __ldcg(p.x_in + (size_t)i * DIM + d) : 0.f;
      if (!isfinite(x)) bad = true;
      v.c[d] = x;
    }
    if (bad) set_error(ctrl, E_NONFINITE);
#pragma unroll
    for (int c = 0; c < 3; ++c) st_acc<DIM>(p.acc + c * vs, i, vzero<DIM>());
    if (p.mode == KM_SOLVE) {
      // the given right-hand side takes the place of L^X X; the CG starts from 0
      stv<DIM>(p.X, i, vzero<DIM>());
      st_acc<DIM>(acc0, i, v);
    } else {
      stv<DIM>(p.X, i, v);
    }
  }
  FD_SYNC(1);

  if (p.mode == KM_ENERGY) {
    if (!pair_pass<DIM, PM_STRESS, 1, CODE, TPS>(p, smem, ps, direct_src(p.X), acc0, RSUM)) return;
    FD_SYNC_RED(2, red_stress(1));
    if (blockIdx.x == 0 && tid == 0) {
      df f[1];
      load_red<1>(ctrl, f);
      const double fd = df_to_double(f[0]);
      ctrl->f_final = fd;
      ctrl->pair_passes = 1.0;
      ctrl->stress_passes = 1.0;
      if (!isfinite(fd)) set_error(ctrl, E_NONFINITE);
    }
    return;
  }

  if (p.mode == KM_FORCES) {
    if (!pair_pass<DIM, PM_FORCES, 1, CODE, TPS>(p, smem, ps, direct_src(p.X), acc0)) return;
    FD_SYNC(3);
    vertex_phase<0>(p, red64, nullptr, [&](int i, df(&)[1]) {
      const Vec<DIM> f = take_acc<DIM>(acc0, i);
      if (i < n) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = f.c[d];
      }
    });
    if (blockIdx.x == 0 && tid == 0) {
      ctrl->pair_passes = 1.0;
      ctrl->stress_passes = 1.0;
    }
    return;
  }

  // ======================= KM_RUN: Algorithm 2 ============================
  // The loop's scalars live in shared memory: thread 0 updates them after
  // each grid barrier and the CTA reads them after a CTA barrier, so that the
  // all-pairs passes keep their registers.  Every CTA computes the same
  // values from the same reductions, so control flow is uniform over the grid.
  RunState* rs = reinterpret_cast<RunState*>(smem + L::OFF_RUN);
#define cgt2 ((float)(p.cg_tol * p.cg_tol))
  // b = L^{X^0} X^0 (right-hand side of Eq. (2-5)) and f(X^0) (Eq. (1));
  // KM_SOLVE has its right-hand side already
  if (p.mode != KM_SOLVE) {
    if (!pair_pass<DIM, PM_RHS, 1, CODE, TPS>(p, smem, ps, direct_src(p.X), acc0, RSUM)) return;
    FD_SYNC_RED(4, red_stress(1));
  }
  if (tid == 0) {
    df f[1];
    if (p.mode != KM_SOLVE) load_red<1>(ctrl, f);
    else f[0] = df_of(0.f);
    const double f0 = df_to_double(f[0]);
    rs->f_cur = rs->f_new = f0;
    rs->crit = 0.0;
    rs->passes_mv = 0.0;
    rs->passes_st = (p.mode != KM_SOLVE) ? 1.0 : 0.0;
    rs->passes_en = 0.0;
    rs->cg_total = rs->cg_maxed = rs->cg_stalled = rs->n_acc = rs->it_outer = 0;
    rs->accept = 0;
    rs->bsel = 0;
    rs->om_prev = 0.f;
    for (int d = 0; d < 3; ++d) rs->z0[d] = 0.f;
    rs->stop = isfinite(f0) ? 0 : 1;
    if (rs->stop) set_error(ctrl, E_NONFINITE);
    if (blockIdx.x == 0 && p.mode != KM_SOLVE) p.trace_f[0] = f0;
  }
  __syncthreads();
  if (rs->stop) return;

  for (int k = 0;; ++k) {
    // ---- start of the H step.  x0 = X^0, or the candidate line 6 kept (formed
    // on the fly from the CG solution and the previous layout); L^W x0.
    // L^W x0 comes from an all-pairs pass at the launch's first iteration and
    // every LWX_REFRESH-th; in between from the previous H step's own
    // vectors, with no pass: its solve ended at z with residual R = B - L^W z
    // (kept by the CG recurrences), and started from X^k with R0 = B - L^W X^k,
    // so L^W z = B - R, L^W X^k = B - R0, and the kept candidate's product is
    // L^W z, or (1 + w_i) L^W z - w_i L^W X^k for the extrapolation of Eq. (10)
    // (L^W 1 = 0: the pin's translation changes nothing).  The recurrence
    // residual drifts from the true one by about FP32 rounding of the CG
    // updates (1e-7 of R per H step), far below the solve tolerance; the
    // periodic pass resets it.  Per-vertex factors (Sec. 6) scale the
    // extrapolation vertex by vertex, and L^W does not commute with that
    // scaling: with factors every H step runs the pass.
    const bool lwx_pass = (k % LWX_REFRESH) == 0 || p.om_scale != nullptr;
    {
      if (lwx_pass) {
        PassSrc src = direct_src(k == 0 ? p.X : p.Zw, k == 0 ? SK_DIRECT : SK_SEL);
        if (k > 0) {
          src.a[1] = p.X;
#pragma unroll
          for (int d = 0; d < DIM; ++d) src.z0[d] = rs->z0[d];
          src.om = rs->om_prev;
          src.sel = rs->accept;
          src.oms = p.om_scale;
        }
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE, TPS>(p, smem, ps, src, acc2)) return;
        if (tid == 0) rs->passes_mv += 1.0;
        FD_SYNC(5);
      }
      // r0 = b - L^W x0, u0 = M^-1 r0, p = s = 0; displacement sums of x0 against X^k.
      // Scalars: [0,D) r.u  [D,2D) r.r  [2D,3D) b.b  [3D,4D) sum dx  [4D,5D) sum dx^2
      //          [5D,6D) sum x  [6D,7D) sum x^2
      const bool first = (k == 0), acc_t = rs->accept != 0, bsel = rs->bsel != 0;
      const float om_p = rs->om_prev;
      const float* oms = p.om_scale;
      float z0[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) z0[d] = rs->z0[d];
      vertex_phase<7 * DIM>(p, red64, RSUM, [&](int i, df(&v)[7 * DIM]) {
        const bool real = i < n;
        const Vec<DIM> xo = ldv<DIM>(p.X, i);
        const float om_i = (!first && oms) ? om_p * __ldg(oms + i) : om_p;  // Sec. 6: omega_i = omega m_i
        Vec<DIM> x0;
        if (first) {
          x0 = xo;
        } else {
          const Vec<DIM> zw = ldv<DIM>(p.Zw, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const float z = zw.c[d] - z0[d];
            x0.c[d] = real ? (acc_t ? sor_xt(z, xo.c[d], om_i) : z) : 0.f;
          }
        }
        const Vec<DIM> bz = take_acc<DIM>(acc0, i);
        const Vec<DIM> bt = take_acc<DIM>(acc1, i);
        const Vec<DIM> b = bsel ? bt : bz;
        const float s = __ldcg(p.s + i), is = __ldcg(p.inv_s + i);
        // L^W x0: from the pass, or from the previous H step's vectors
        Vec<DIM> lwx;
        if (lwx_pass) {
          const Vec<DIM> a = take_acc<DIM>(acc2, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) lwx.c[d] = fmaf(s, x0.c[d], -a.c[d]);
        } else {
          const Vec<DIM> bk = ldv<DIM>(p.B, i), rf = ldv<DIM>(p.R, i), r0 = ldv<DIM>(p.R0, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const float lz = bk.c[d] - rf.c[d];
            lwx.c[d] = acc_t ? fmaf(1.f + om_i, lz, -om_i * (bk.c[d] - r0.c[d])) : lz;
          }
        }
        Vec<DIM> r, u;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          r.c[d] = b.c[d] - lwx.c[d];
          u.c[d] = is * r.c[d];
          const df dx = real ? df_diff(x0.c[d], xo.c[d]) : df_of(0.f);
          const float xv = real ? x0.c[d] : 0.f;
          v[d] = df_add(v[d], df_prod(r.c[d], u.c[d]));
          v[DIM + d] = df_add(v[DIM + d], df_prod(r.c[d], r.c[d]));
          v[2 * DIM + d] = df_add(v[2 * DIM + d], df_prod(b.c[d], b.c[d]));
          v[3 * DIM + d] = df_add(v[3 * DIM + d], dx);
          v[4 * DIM + d] = df_add(v[4 * DIM + d], df_sqr(dx));
          v[5 * DIM + d] = df_add(v[5 * DIM + d], df_of(xv));
          v[6 * DIM + d] = df_add(v[6 * DIM + d], df_prod(xv, xv));
        }
        stv<DIM>(p.Zw, i, x0);
        stv<DIM>(p.X, i, x0);
        stv<DIM>(p.R, i, r);
        stv<DIM>(p.R0, i, r);
        stv<DIM>(p.B, i, b);
        stv<DIM>(p.U, i, u);
        stv<DIM>(p.P, i, vzero<DIM>());
        stv<DIM>(p.S, i, vzero<DIM>());
      });
      // reduce the 7*DIM sums; the last CTA also evaluates the termination rule
      const double fcur_k = rs->f_cur, fnew_k = rs->f_new;
      auto red_init = [&](const double* sums) {
        take_sums<7 * DIM>(ctrl, sums);
        if (threadIdx.x == 0) {
          double c = 0.0;
          if (p.stop == 0) {
            double num = 0.0, den = 0.0;
            for (int d = 0; d < DIM; ++d) {
              const float2 a1 = ctrl->red[3 * DIM + d], a2 = ctrl->red[4 * DIM + d];
              const float2 a3 = ctrl->red[5 * DIM + d], a4 = ctrl->red[6 * DIM + d];
              const double s1 = (double)a1.x + a1.y, s2 = (double)a2.x + a2.y;
              const double x1 = (double)a3.x + a3.y, x2 = (double)a4.x + a4.y;
              num += fmax(s2 - s1 * s1 / n, 0.0);
              den += fmax(x2 - x1 * x1 / n, 0.0);
            }
            c = (den > 0.0) ? sqrt(num / den) : 0.0;
          } else {
            c = (fcur_k != 0.0) ? (fcur_k - fnew_k) / fcur_k : 0.0;
          }
          ctrl->red_d[0] = c;
        }
      };
      FD_SYNC_RED(9, red_init);
      if (tid == 0) {
        df v[3 * DIM];
        load_red<3 * DIM>(ctrl, v);
        int all = 1;
        for (int d = 0; d < DIM; ++d) {
          rs->rz[d] = df_f(v[d]);
          const float rr = df_f(v[DIM + d]);
          rs->bb[d] = df_f(v[2 * DIM + d]);
          rs->conv[d] = (rr <= cgt2 * rs->bb[d]) ? 1 : 0;
          all = all && rs->conv[d];
        }
        rs->all_conv = all;
        rs->it = 0;
        rs->stop = 0;
        if (k > 0) {
          const double crit = __ldcg(&ctrl->red_d[0]);
          rs->crit = crit;
          if (blockIdx.x == 0) p.trace_crit[k - 1] = crit;
          rs->f_cur = rs->f_new;
          rs->it_outer = k;
          rs->stop = (crit < p.tol || k >= p.max_iter) ? 1 : 0;
        }
      }
      __syncthreads();
      if (rs->stop) break;
    }
    if (p.solver == SOLVER_DIRECT) {
      // ---- refinement with the factored inverse: delta = A'^-1 r, x += delta,
      // r -= L^W delta (pair pass), until every column meets cg_tol or cg_max
      // steps ran.  r sums to zero (b = L^X X does, L^W x does), so A'^-1 r
      // is the minimum-norm solution of L^W delta = r.
      float* dbuf = reinterpret_cast<float*>(smem + L::stage_base(CODE == CODE_U8 ? p.lut_rows * LUT_ROW : 0));
      while (!rs->all_conv) {
        // delta goes to P (unused by this solver; zeroed at the start of the H
        // step and by every refinement's vertex phase)
        dense_apply<DIM>(p, dbuf, p.R, p.P);
        FD_SYNC(10);
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE, TPS>(p, smem, ps, direct_src(p.P), acc2)) return;
        if (tid == 0) {
          rs->passes_mv += 1.0;
          ++rs->it;
        }
        FD_SYNC(7);
        vertex_phase<DIM>(p, red64, RSUM, [&](int i, df(&v)[DIM]) {
          const float s = __ldcg(p.s + i);
          const Vec<DIM> u = take_acc<DIM>(p.P, i);
          const Vec<DIM> a = take_acc<DIM>(acc2, i);
          Vec<DIM> x = ldv<DIM>(p.Zw, i), r = ldv<DIM>(p.R, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            x.c[d] += u.c[d];
            r.c[d] -= fmaf(s, u.c[d], -a.c[d]);
            v[d] = df_add(v[d], df_prod(r.c[d], r.c[d]));
          }
          stv<DIM>(p.Zw, i, x);
          stv<DIM>(p.R, i, r);
        });
        auto red_dir = [&](const double* sums) { take_sums<DIM>(ctrl, sums); };
        FD_SYNC_RED(9, red_dir);
        if (tid == 0) {
          df v[DIM];
          load_red<DIM>(ctrl, v);
          int all = 1;
          for (int d = 0; d < DIM; ++d) {
            if (!rs->conv[d]) rs->conv[d] = (df_f(v[d]) <= cgt2 * rs->bb[d]) ? 1 : 0;
            all = all && rs->conv[d];
          }
          if (!all && rs->it >= p.cg_max) {
            ++rs->cg_maxed;
            all = 1;
          }
          rs->all_conv = all;
        }
        __syncthreads();
      }
    }
    // ---- CG on L^W Z = b, one reduction per step
    if (p.solver != SOLVER_DIRECT && !rs->all_conv) {
      if (!pair_pass<DIM, PM_MATVEC, 1, CODE, TPS>(p, smem, ps, direct_src(p.U), acc2)) return;
      if (tid == 0) rs->passes_mv += 1.0;
      FD_SYNC(6);
      // w0 = L^W u0 and delta0 = (w0, u0).  Slots [0,D).
      vertex_phase<DIM>(p, red64, RSUM, [&](int i, df(&v)[DIM]) {
        const float s = __ldcg(p.s + i);
        const Vec<DIM> u = ldv<DIM>(p.U, i);
        const Vec<DIM> a = take_acc<DIM>(acc2, i);
        Vec<DIM> w;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          w.c[d] = fmaf(s, u.c[d], -a.c[d]);
          v[d] = df_add(v[d], df_prod(w.c[d], u.c[d]));
        }
        stv<DIM>(p.W, i, w);
      });
      auto red_au0 = [&](const double* sums) { take_sums<DIM>(ctrl, sums); };
      FD_SYNC_RED(9, red_au0);
      if (tid == 0) {
        df dlv[DIM];
        load_red<DIM>(ctrl, dlv);
        for (int d = 0; d < DIM; ++d) {
          const float dl = df_f(dlv[d]);
          rs->gam[d] = rs->rz[d];
          rs->beta[d] = 0.f;
          if (!rs->conv[d] && !(dl > 0.f)) {
            rs->conv[d] = 1;  // u0 carries no curvature: nothing to solve in this column
            ++rs->cg_stalled;
          }
          rs->alpha[d] = rs->conv[d] ? 0.f : rs->gam[d] / dl;
        }
      }
      __syncthreads();
      if (tid == 0) rs->cg_last = 0;
      __syncthreads();
      while (true) {
        // One step of preconditioned CG in the single-reduction form of
        // Chronopoulos and Gear: p = u + beta p, s = w + beta s, x += alpha p,
        // r -= alpha s, u = M^-1 r, w = L^W u.  The curvature (p', L^W p') of
        // the next direction p' = u + beta' p is needed before beta' is known;
        // it is expanded as (u,w) + beta' ((u,s) + (p,w)) + beta'^2 (p,s) from
        // dot products taken here, instead of the usual recurrence, which
        // loses positivity in FP32.  The pass of a step computes w for the
        // step after it; when the residual that step leaves, expanded as
        // |r - alpha (w + beta s)|^2 from dot products taken here too, already
        // meets cg_tol, the step runs without its pass (cg_last) and ends the
        // solve: that pass's w would never be used.
        // Slots: [0,D) r.u  [D,2D) w.u  [2D,3D) r.r  [3D,4D) u.s  [4D,5D) p.w  [5D,6D) p.s
        //        [6D,7D) r.w  [7D,8D) r.s  [8D,9D) w.w  [9D,10D) w.s  [10D,11D) s.s
        if (rs->cg_last) {
          float al[DIM], be[DIM];
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            al[d] = rs->alpha[d];
            be[d] = rs->beta[d];
          }
          vertex_phase<0>(p, red64, nullptr, [&](int i, df(&)[1]) {
            const Vec<DIM> u = ldv<DIM>(p.U, i), w = ldv<DIM>(p.W, i), pp = ldv<DIM>(p.P, i),
                           sp = ldv<DIM>(p.S, i);
            Vec<DIM> x = ldv<DIM>(p.Zw, i), r = ldv<DIM>(p.R, i);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              x.c[d] = fmaf(al[d], fmaf(be[d], pp.c[d], u.c[d]), x.c[d]);
              r.c[d] = fmaf(-al[d], fmaf(be[d], sp.c[d], w.c[d]), r.c[d]);
            }
            stv<DIM>(p.Zw, i, x);
            stv<DIM>(p.R, i, r);
          });
          if (tid == 0) ++rs->it;
          FD_SYNC(12);
          break;
        }
        PassSrc src = direct_src(p.R, SK_CGU);
        src.a[1] = p.W;
        src.a[2] = p.S;
        src.a[3] = p.inv_s;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          src.alpha[d] = rs->alpha[d];
          src.beta[d] = rs->beta[d];
        }
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE, TPS>(p, smem, ps, src, acc2)) return;
        if (tid == 0) {
          rs->passes_mv += 1.0;
          ++rs->it;
        }
        FD_SYNC(7);
        float al[DIM], be[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          al[d] = src.alpha[d];
          be[d] = src.beta[d];
        }
        // 11 D sums: more than the reduction scratch at OFF_RED64 holds in 3-D;
        // the stage area is idle between passes and takes them
        float2* red_cg_buf = reinterpret_cast<float2*>(smem + L::stage_base(CODE == CODE_U8 ? p.lut_rows * LUT_ROW : 0));
        vertex_phase<11 * DIM>(p, red_cg_buf, RSUM, [&](int i, df(&v)[11 * DIM]) {
          const float s = __ldcg(p.s + i), is = __ldcg(p.inv_s + i);
          Vec<DIM> u = ldv<DIM>(p.U, i), w = ldv<DIM>(p.W, i), pp = ldv<DIM>(p.P, i), sp = ldv<DIM>(p.S, i);
          Vec<DIM> x = ldv<DIM>(p.Zw, i), r = ldv<DIM>(p.R, i);
          const Vec<DIM> a = take_acc<DIM>(acc2, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const float pn = fmaf(be[d], pp.c[d], u.c[d]);
            const float sn = fmaf(be[d], sp.c[d], w.c[d]);
            const float un = cg_u(r.c[d], w.c[d], sp.c[d], is, al[d], be[d]);
            x.c[d] = fmaf(al[d], pn, x.c[d]);
            r.c[d] = fmaf(-al[d], sn, r.c[d]);
            pp.c[d] = pn;
            sp.c[d] = sn;
            u.c[d] = un;
            w.c[d] = fmaf(s, un, -a.c[d]);
            v[d] = df_add(v[d], df_prod(r.c[d], un));
            v[DIM + d] = df_add(v[DIM + d], df_prod(w.c[d], un));
            v[2 * DIM + d] = df_add(v[2 * DIM + d], df_prod(r.c[d], r.c[d]));
            v[3 * DIM + d] = df_add(v[3 * DIM + d], df_prod(un, sn));
            v[4 * DIM + d] = df_add(v[4 * DIM + d], df_prod(pn, w.c[d]));
            v[5 * DIM + d] = df_add(v[5 * DIM + d], df_prod(pn, sn));
            v[6 * DIM + d] = df_add(v[6 * DIM + d], df_prod(r.c[d], w.c[d]));
            v[7 * DIM + d] = df_add(v[7 * DIM + d], df_prod(r.c[d], sn));
            v[8 * DIM + d] = df_add(v[8 * DIM + d], df_prod(w.c[d], w.c[d]));
            v[9 * DIM + d] = df_add(v[9 * DIM + d], df_prod(w.c[d], sn));
            v[10 * DIM + d] = df_add(v[10 * DIM + d], df_prod(sn, sn));
          }
          stv<DIM>(p.P, i, pp);
          stv<DIM>(p.S, i, sp);
          stv<DIM>(p.Zw, i, x);
          stv<DIM>(p.R, i, r);
          stv<DIM>(p.U, i, u);
          stv<DIM>(p.W, i, w);
        });
        auto red_cg = [&](const double* sums) { take_sums<11 * DIM>(ctrl, sums); };
        FD_SYNC_RED(9, red_cg);
        if (tid == 0) {
          df v[11 * DIM];
          load_red<11 * DIM>(ctrl, v);
          int done = 1;
          for (int d = 0; d < DIM; ++d) {
            const float gn = df_f(v[d]), dn = df_f(v[DIM + d]), rrn = df_f(v[2 * DIM + d]);
            if (!rs->conv[d]) {
              rs->conv[d] = (rrn <= cgt2 * rs->bb[d]) ? 1 : 0;
              if (!rs->conv[d]) {
                const float bn = gn / rs->gam[d];
                const float pi =
                    dn + bn * (df_f(v[3 * DIM + d]) + df_f(v[4 * DIM + d])) + bn * bn * df_f(v[5 * DIM + d]);
                if (pi > 0.f && gn > 0.f) {
                  rs->beta[d] = bn;
                  rs->alpha[d] = gn / pi;
                } else {
                  rs->conv[d] = 1;  // curvature lost to rounding: the solve has gone as far as FP32 allows
                  ++rs->cg_stalled;
                }
              }
              if (rs->conv[d]) {
                rs->alpha[d] = 0.f;
                rs->beta[d] = 0.f;
              }
            }
            rs->gam[d] = gn;
            done = done && rs->conv[d];
          }
          if (!done && rs->it >= p.cg_max) {
            ++rs->cg_maxed;
            done = 1;
          }
          rs->cg_done = done;
          if (!done) {
            // the residual after the next update, r' = r - alpha (w + beta s), per
            // column: if every column meets cg_tol with it, the next step is the
            // last and needs no pass
            int last = 1;
            for (int d = 0; d < DIM; ++d) {
              if (rs->conv[d]) continue;
              const double al = rs->alpha[d], be = rs->beta[d];
              const double rr = df_to_double(v[2 * DIM + d]);
              const double rs_ = df_to_double(v[6 * DIM + d]) + be * df_to_double(v[7 * DIM + d]);
              const double ss = df_to_double(v[8 * DIM + d]) + 2.0 * be * df_to_double(v[9 * DIM + d]) +
                                be * be * df_to_double(v[10 * DIM + d]);
              const double rr_next = rr - 2.0 * al * rs_ + al * al * ss;
              if (!(rr_next <= (double)cgt2 * (double)rs->bb[d])) last = 0;
            }
            rs->cg_last = last;
          }
        }
        __syncthreads();
        if (rs->cg_done) break;
      }
    }

    if (p.mode == KM_SOLVE) {
      // Y = the CG solution with vertex 0 moved to the origin (Sec. 2 after Prop. 2.3)
      const Vec<DIM> zz = ldv<DIM>(p.Zw, 0);
      for (int R = blockIdx.x; R < nb; R += gridDim.x) {
        const int i = R * TILE + tid;
        if (i < n) {
          const Vec<DIM> z = ldv<DIM>(p.Zw, i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = z.c[d] - zz.c[d];
        }
      }
      if (blockIdx.x == 0 && tid == 0) {
        ctrl->iters = 0;
        ctrl->cg_steps = rs->it;
        ctrl->cg_maxed = rs->cg_maxed;
        ctrl->cg_stalled = rs->cg_stalled;
        ctrl->pair_passes = rs->passes_mv;
        ctrl->matvec_passes = rs->passes_mv;
        ctrl->stress_passes = 0.0;
      }
      return;
    }
    if (WITH_ENUM && p.enum_omega) {
      // ---- enumerating strategy (Sec. 5.2.2): the stress of every
      // (1 + omega) z - omega x, omega in {0, 0.5, ..., 9}, from one pass; the
      // argmin (ties to the smaller omega) becomes X^{k+1}, and a second pass
      // gives its right-hand side and stress.
      PassSrc src = direct_src(p.Zw, SK_ZX);
      src.a[1] = p.X;
      src.oms = p.om_scale;
      const Vec<DIM> zz = ldv<DIM>(p.Zw, 0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) src.z0[d] = zz.c[d];
      __syncthreads();  // every thread has read the scalars of this iteration
      if (tid == 0) {
        rs->cg_total += rs->it;
        for (int d = 0; d < DIM; ++d) rs->z0[d] = src.z0[d];
        rs->passes_en += (double)NENUM;  // the enumeration pass: NENUM stresses, no right-hand side
        rs->passes_st += 1.0;            // the pass on the selected candidate
      }
      if constexpr (WITH_ENUM) {
        if (!pair_pass<DIM, PM_ENUM, 2, CODE, TPS>(p, smem, ps, src, acc0, RSUM)) return;
      }
      auto red_enum = [&](const double* sums) { take_sums<NENUM>(ctrl, sums); };
      FD_SYNC_RED(8, red_enum);
      if (tid == 0) {
        df fv[NENUM];
        load_red<NENUM>(ctrl, fv);
        int best = 0;
        double fbest = df_to_double(fv[0]);
        for (int e = 1; e < NENUM; ++e) {
          const double fe = df_to_double(fv[e]);
          if (fe < fbest) {
            fbest = fe;
            best = e;
          }
        }
        rs->om_prev = ENUM_STEP * best;
        rs->accept = (best > 0) ? 1 : 0;
        rs->bsel = 0;
        rs->f_enum0 = df_to_double(fv[0]);
      }
      __syncthreads();
      PassSrc sel = direct_src(p.Zw, SK_SEL);
      sel.a[1] = p.X;
#pragma unroll
      for (int d = 0; d < DIM; ++d) sel.z0[d] = src.z0[d];
      sel.om = rs->om_prev;
      sel.sel = rs->accept;
      sel.oms = p.om_scale;
      if (!pair_pass<DIM, PM_RHS, 1, CODE, TPS>(p, smem, ps, sel, acc0, RSUM)) return;
      FD_SYNC_RED(8, red_stress(1));
      if (tid == 0) {
        df fz[1];
        load_red<1>(ctrl, fz);
        const double fX = df_to_double(fz[0]);
        if (!isfinite(fX)) {
          set_error(ctrl, E_NONFINITE);
          rs->stop = 1;
        } else {
          rs->f_new = fX;
          if (rs->accept) ++rs->n_acc;
          if (blockIdx.x == 0) {
            p.trace_f[k + 1] = fX;
            p.trace_acc[k] = rs->accept;
            p.trace_om[k] = (double)rs->om_prev;
            p.trace_cg[k] = rs->it;
            p.trace_fh[k] = rs->f_enum0;
            p.trace_ft[k] = fX;
            p.trace_t[k] = 1e-6 * (double)(globaltimer_ns() - t_launch);
          }
        }
      }
      __syncthreads();
      if (rs->stop) return;
      continue;
    }
    // ---- pin vertex 0 (Sec. 2), extrapolate (Eq. (10)), stress and RHS of both candidates
    const double om = p.omega_seq[k];
    const bool two = (om != 0.0);
    PassSrc src = direct_src(p.Zw, SK_K2);
    src.a[1] = p.X;
    src.oms = p.om_scale;
    {
      const Vec<DIM> zz = ldv<DIM>(p.Zw, 0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) src.z0[d] = zz.c[d];
      src.om = (float)om;
    }
    __syncthreads();  // every thread has read the scalars of this iteration
    if (tid == 0) {
      rs->cg_total += rs->it;
      for (int d = 0; d < DIM; ++d) rs->z0[d] = src.z0[d];
      rs->om_prev = src.om;
      rs->passes_st += two ? 2.0 : 1.0;
    }
    // Both candidates' stresses, and the right-hand side of the extrapolated
    // one only: line 6 keeps it in most iterations; when it keeps z instead, a
    // pass for z's right-hand side follows (below).
    if (two) {
      if (!pair_pass<DIM, PM_K2L, 2, CODE, TPS>(p, smem, ps, src, acc0, RSUM)) return;
      FD_SYNC_RED(8, red_stress(2));
    } else {
      if (!pair_pass<DIM, PM_RHS, 1, CODE, TPS>(p, smem, ps, src, acc0, RSUM)) return;
      FD_SYNC_RED(8, red_stress(1));
    }
    if (tid == 0) {
      df fz[2];
      load_red<2>(ctrl, fz);
      const double fZ = df_to_double(fz[0]);
      const double fT = two ? df_to_double(fz[1]) : fZ;
      if (two && blockIdx.x == 0) ctrl->rhs_skipped += 1.0;
      if (!isfinite(fZ) || !isfinite(fT)) {
        set_error(ctrl, E_NONFINITE);
        rs->stop = 1;
      } else {
        // line 6 (ties accept).  With omega = 0 the two candidates coincide and
        // X^{k+1} is kept as it is (the test is trivially true).
        const bool accept = two && (fT <= fZ);
        rs->accept = accept ? 1 : 0;
        rs->bsel = rs->accept;
        rs->f_new = accept ? fT : fZ;
        if (accept || !two) ++rs->n_acc;
        if (blockIdx.x == 0) {
          p.trace_f[k + 1] = rs->f_new;
          p.trace_acc[k] = (accept || !two) ? 1 : 0;
          p.trace_om[k] = om;
          p.trace_cg[k] = rs->it;
          p.trace_fh[k] = fZ;
          p.trace_ft[k] = fT;
          p.trace_t[k] = 1e-6 * (double)(globaltimer_ns() - t_launch);
        }
      }
    }
    __syncthreads();
    if (rs->stop) return;
    if (two && !rs->accept) {
      // z is kept: its right-hand side, which the two-candidate pass left out
      // (this pass recomputes z's stress; that value is not used)
      PassSrc zs = direct_src(p.Zw, SK_SEL);
      zs.a[1] = p.X;
#pragma unroll
      for (int d = 0; d < DIM; ++d) zs.z0[d] = src.z0[d];
      zs.om = src.om;
      zs.sel = 0;
      zs.oms = p.om_scale;
      if (!pair_pass<DIM, PM_RHS, 1, CODE, TPS>(p, smem, ps, zs, acc0, RSUM)) return;
      if (tid == 0) rs->passes_st += 1.0;
      FD_SYNC_RED(11, red_stress(1));
    }
  }

  // --- output: X holds the layout accepted by the last iteration
  for (int R = blockIdx.x; R < nb; R += gridDim.x) {
    const int i = R * TILE + tid;
    if (i < n) {
      const Vec<DIM> x = ldv<DIM>(p.X, i);
#pragma unroll
      for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = x.c[d];
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    ctrl->iters = rs->it_outer;
    ctrl->cg_steps = rs->cg_total;
    ctrl->cg_maxed = rs->cg_maxed;
    ctrl->cg_stalled = rs->cg_stalled;
    ctrl->accepted = rs->n_acc;
    ctrl->f_final = rs->f_cur;
    ctrl->crit_final = rs->crit;
    ctrl->pair_passes = rs->passes_mv + rs->passes_st + rs->passes_en;
    ctrl->matvec_passes = rs->passes_mv;
    ctrl->stress_passes = rs->passes_st;
    ctrl->enum_passes = rs->passes_en;
  }
#undef FD_SYNC
#undef FD_SYNC_RED
#undef RSUM
#undef n
#undef nb
#undef tid
#undef vs
#undef acc0
#undef acc1
#undef acc2
#undef red64
#undef ctrl
#undef cgt2
}

}  // namespace fdl
