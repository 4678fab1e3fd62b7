// fd_solver.cuh -- the cooperative layout kernel (stress, forces, and the
// whole Algorithm 2 loop of Wang & Wang 2012) for one layout dimension and
// one distance-code type.  Included by fd_solver_d{1,2,3}.cu.
//
// Work decomposition
// ------------------
// All-pairs passes run over the tiles of the half ring (fd_internal.cuh),
// grouped into tasks of consecutive tiles of one block row.  CTAs take tasks
// from a global ticket counter.  A CTA has 4 warps; every warp holds all 128
// rows of block I (4 rows per lane, in registers) and sweeps 32 columns of
// block J.  In step t lane l pairs its 4 rows with column 32w + ((l + t) & 31);
// the column accumulators travel one lane down after every step, so after 32
// steps each lane holds the complete column sums of its own column and both
// endpoints of every pair are accumulated exactly once (symmetric n-body).
//
// Pipeline: a tile's distance codes (16 KB for uint8) and the raw per-vertex
// arrays of its two blocks arrive by 1-D bulk copies (TMA) on one mbarrier,
// issued one tile ahead.  The raw arrays are turned into the pass's vectors
// in shared memory (e.g. the CG vector u = M^-1 (r - alpha s) is formed on
// the fly), so every pass reads only what the previous pass left in memory.
// CTA b takes tasks b, b + G, b + 2G, ... (G CTAs): a pass has no global
// synchronisation inside it.
//
// Reductions: per-tile column partials and per-task row partials go to
// global buffers.  After the pass (grid barrier) one CTA per row block sums
// its partials in a fixed order (Kahan-compensated) and runs the step's
// per-row epilogue, which updates the vectors in place.  Scalars (stress,
// CG dot products, displacement sums) are FP64 sums in a fixed order;
// results never depend on timing.
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

enum PairMode { PM_STRESS = 0, PM_FORCES = 1, PM_RHS = 2, PM_MATVEC = 3 };

// How a pass forms its vectors from the raw arrays it copies.
enum SrcKind {
  SK_DIRECT = 0,  // v = a[0]
  SK_CGU = 1,     // u = inv_s * (r - alpha * (w + beta * s_prev)); a = {r, w, s_prev, inv_s}
  SK_K2 = 2       // z = zw - zw_0, xt = (1 + omega) z - omega x; a = {zw, x}
};

template <int SK>
struct SrcN {
  static constexpr int v = (SK == SK_DIRECT) ? 1 : (SK == SK_CGU) ? 4 : 2;
};

struct PassSrc {
  const float* a[4];
  float alpha[3], beta[3];  // SK_CGU, per column
  float z0[3];              // SK_K2: pinned vertex 0 of the CG solution
  float om;                 // SK_K2: omega of Eq. (10)
};

// The CG vector u_{i+1} (used both on the fly and in the epilogue, so that
// the two agree bit for bit).
__device__ __forceinline__ float cg_u(float r, float w, float sp, float is, float alpha, float beta) {
  return is * fmaf(-alpha, fmaf(beta, sp, w), r);
}
// Eq. (10): X~ = (1 + omega) X^{k+1} - omega X^k.
__device__ __forceinline__ float sor_xt(float z, float x, float om) { return fmaf(1.0f + om, z, -(om * x)); }

template <int CODE>
struct CodeBytes {
  static constexpr int v = (CODE == CODE_U8) ? 1 : 4;
};

// Shared memory.  The lookup table is replicated so that every lane reads
// its own bank: row c (256 bytes) holds 32 copies of 1/d^2 (bytes 0..127)
// and 16 copies of {1/d, -1} (bytes 128..255) for code c.
template <int DIM, int CODE>
struct SmemLayout {
  static constexpr int DP = DimP<DIM>::v;
  static constexpr int DBUF = TILE * TILE * CodeBytes<CODE>::v;
  static constexpr int RAW_ARR = TILE * DP * 4;                  // bytes of one block of one raw array
  static constexpr int OFF_RED64 = 0;                            // float2 [CTA] reduction scratch
  static constexpr int OFF_IDX = OFF_RED64 + CTA * 8;            // int [CTA] contribution indices
  static constexpr int OFF_MISC = OFF_IDX + CTA * 4;             // mbar[2], slots
  static constexpr int OFF_POSI = 2048;                          // [2][TILE][DP], row-interleaved
  static constexpr int OFF_POSJ = OFF_POSI + 2 * RAW_ARR;        // [2][TILE][DP]
  static constexpr int OFF_RAW = OFF_POSJ + 2 * RAW_ARR;         // [4 arrays][2 blocks][TILE][DP] floats
  static constexpr int OFF_D0 = ((OFF_RAW + 4 * 2 * RAW_ARR + 127) / 128) * 128;
  static constexpr int OFF_D1 = OFF_D0 + DBUF;
  static constexpr int OFF_LUT = ((OFF_D1 + DBUF + 255) / 256) * 256;
  static constexpr int BASE_BYTES = OFF_LUT;
  static_assert(OFF_MISC + 64 <= OFF_POSI, "fixed regions overlap");
  static_assert(4 * 2 * TILE * DP * 4 <= DBUF, "row partial area must fit in a distance buffer");
};
constexpr int SMEM_OFF_IDX = CTA * 8;  // OFF_IDX, identical for every layout
constexpr int SMEM_OFF_POSI = 2048;   // OFF_POSI, identical for every layout

struct PairState {
  unsigned parity;  // bit b: phase parity of mbarrier b
  int pass;         // passes run so far (selects the scalar buffer parity)
};

// --------------------------------------------------------------------------
// Deterministic FP64 reductions
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

// Sums slots [off, off+K) of the row-block scalar array (stride per block)
// over nb blocks; every CTA gets the identical values.
template <int K>
__device__ __forceinline__ void sum_blocks(const float2* a, int nb, int stride, int off, df (&out)[K], float2* red) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = df_of(0.f);
  for (int R = threadIdx.x; R < nb; R += CTA) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = df_add(out[k], df_ld(a + (size_t)R * stride + off + k));
  }
  cta_sum_multi<K>(out, red);
}
__device__ __forceinline__ float df_f(df a) { return a.hi + a.lo; }

// Sum of the per-CTA stress slots (candidate c) in a fixed order.
__device__ __forceinline__ double sum_ctas(const float2* sc, int c, float2* red) {
  df v[1] = {df_of(0.f)};
  for (int t = threadIdx.x; t < (int)gridDim.x; t += CTA) v[0] = df_add(v[0], df_ld(sc + (size_t)t * 2 + c));
  cta_sum_multi<1>(v, red);
  return df_to_double(v[0]);
}

// Grid barrier whose last arriving CTA runs `on_last` (all its threads)
// before it releases the others: reductions over all CTAs' partial sums run
// once, in a fixed order, instead of in every CTA.  Waits are bounded.
template <class F>
__device__ __forceinline__ bool grid_sync_reduce(Ctrl* c, long long timeout_ns, int where, F&& on_last) {
  __shared__ int s_last, s_ok;
  __syncthreads();
  unsigned int g = 0;
  if (threadIdx.x == 0) {
    g = *(volatile unsigned int*)&c->bar_gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->bar_count, 1u);
    s_last = (arrived == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (s_last) {
    on_last();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned int* gen = &c->bar_gen;
    volatile int* err = &c->err;
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
  if (threadIdx.x == 0) {
    __threadfence();
    s_ok = (*(volatile int*)&c->err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Run by the last CTA: K consecutive slots of `count` records (stride float2
// apart) summed in a fixed order into ctrl->red[0..K).
template <int K>
__device__ __forceinline__ void reduce_slots_to_ctrl(Ctrl* c, const float2* a, int count, int stride, float2* red) {
  df t[K];
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = df_of(0.f);
  for (int r = threadIdx.x; r < count; r += CTA) {
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = df_add(t[k], df_ld(a + (size_t)r * stride + k));
  }
  cta_sum_multi<K>(t, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) __stcg(&c->red[k], make_float2(t[k].hi, t[k].lo));
  }
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

// Independent column-accumulator chains per warp.  Chain c serves the steps
// t = c (mod CH) and travels CH lanes per use, so consecutive steps do not
// wait on each other's shuffles.
template <int MODE, int DIM>
struct Chains {
  static constexpr int v = (MODE == PM_MATVEC) ? 4 : (DIM == 3 ? 1 : 2);
};

template <int DIM, int MODE, int NC, int CODE>
__device__ __forceinline__ void tile_compute(const unsigned char* __restrict__ dt, const float* __restrict__ posj,
                                             const unsigned char* __restrict__ lut,
                                             const Vec<DIM> (&xi)[NC][ROWS_PER_LANE],
                                             Vec<DIM> (&iacc)[NC][ROWS_PER_LANE], Vec<DIM> (&jout)[NC],
                                             float (&st)[NC], int lane, int warp) {
  constexpr int DP = DimP<DIM>::v;
  constexpr int CH = Chains<MODE, DIM>::v;
  constexpr float TINY = 1e-30f;  // keeps rsqrt finite for coincident points; below FP32 resolution of r^2
  const unsigned off_w = 4u * lane;                // this lane's copy of 1/d^2
  const unsigned off_k = 128u + 8u * (lane & 15);  // this lane's copy of {1/d, -1}
  Vec<DIM> jacc[CH][NC];
#pragma unroll
  for (int h = 0; h < CH; ++h)
#pragma unroll
    for (int c = 0; c < NC; ++c) jacc[h][c] = vzero<DIM>();
#pragma unroll 1
  for (int t0 = 0; t0 < 32; t0 += CH) {
#pragma unroll
  for (int h = 0; h < CH; ++h) {
    const int jl = warp * 32 + ((lane + t0 + h) & 31);
    unsigned codes = 0;
    float dv[ROWS_PER_LANE];
    if constexpr (CODE == CODE_U8) {
      codes = *reinterpret_cast<const unsigned*>(dt + jl * TILE + ROWS_PER_LANE * lane);
    } else {
      const float4 q = *reinterpret_cast<const float4*>(dt + 4 * (jl * TILE + ROWS_PER_LANE * lane));
      dv[0] = q.x;
      dv[1] = q.y;
      dv[2] = q.z;
      dv[3] = q.w;
    }
    Vec<DIM> pj[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) pj[c] = lds_v<DIM>(posj + c * TILE * DP, jl);
#pragma unroll
    for (int a = 0; a < ROWS_PER_LANE; ++a) {
      float invd = 0.f, negm = 0.f, w = 0.f;
      if constexpr (CODE == CODE_U8) {
        // byte offset 256 * code + this lane's offset, built by one byte permute
        if constexpr (MODE == PM_MATVEC || MODE == PM_FORCES) {
          const unsigned ow = __byte_perm(codes, off_w, 0x5504u | (unsigned)(a << 4));
          w = *reinterpret_cast<const float*>(lut + ow);
        }
        if constexpr (MODE != PM_MATVEC) {
          const unsigned ok = __byte_perm(codes, off_k, 0x5504u | (unsigned)(a << 4));
          const float2 l = *reinterpret_cast<const float2*>(lut + ok);
          invd = l.x;
          negm = l.y;
        }
      } else {
        const float d = dv[a];
        invd = d > 0.f ? __frcp_rn(d) : 0.f;
        negm = d > 0.f ? -1.f : 0.f;
        w = invd * invd;
      }
      if constexpr (MODE == PM_MATVEC) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          iacc[0][a].c[d] = fmaf(-w, pj[0].c[d], iacc[0][a].c[d]);
          jacc[h][0].c[d] = fmaf(-w, xi[0][a].c[d], jacc[h][0].c[d]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float dx[DIM];
          float r2 = TINY;
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            dx[d] = xi[c][a].c[d] - pj[c].c[d];
            r2 = fmaf(dx[d], dx[d], r2);
          }
          const float rs = rsqrt_approx(r2);
          if constexpr (MODE == PM_STRESS || MODE == PM_RHS) {
            const float r = r2 * rs;
            const float tt = fmaf(r, invd, negm);
            st[c] = fmaf(tt, tt, st[c]);
          }
          if constexpr (MODE == PM_RHS || MODE == PM_FORCES) {
            float coef;
            if constexpr (MODE == PM_RHS) {
              coef = rs * invd;
            } else {
              coef = fmaf(invd, rs, -w);
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              iacc[c][a].c[d] = fmaf(coef, dx[d], iacc[c][a].c[d]);
              jacc[h][c].c[d] = fmaf(-coef, dx[d], jacc[h][c].c[d]);
            }
          }
        }
      }
    }
    if constexpr (MODE != PM_STRESS) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          jacc[h][c].c[d] = __shfl_sync(0xffffffffu, jacc[h][c].c[d], (lane + CH) & 31);
    }
  }
  }
  // chain h of lane l now holds column (l + h) & 31: gather column l's chains
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    jout[c] = jacc[0][c];
#pragma unroll
    for (int h = 1; h < CH; ++h)
#pragma unroll
      for (int d = 0; d < DIM; ++d) jout[c].c[d] += __shfl_sync(0xffffffffu, jacc[h][c].c[d], (lane - h) & 31);
  }
}

// Forms element t of one block (side 0 = I, 1 = J) of the pass's vectors
// from the raw arrays in shared memory.
template <int DIM, int SK, int NC>
__device__ __forceinline__ void form(const PassSrc& s, const float* raw, int side, int t, Vec<DIM> (&out)[NC]) {
  constexpr int DP = DimP<DIM>::v;
  constexpr int A = TILE * DP;  // floats per raw block
  if constexpr (SK == SK_DIRECT) {
    out[0] = lds_v<DIM>(raw + (0 * 2 + side) * A, t);
  } else if constexpr (SK == SK_CGU) {
    const Vec<DIM> r = lds_v<DIM>(raw + (0 * 2 + side) * A, t);
    const Vec<DIM> w = lds_v<DIM>(raw + (1 * 2 + side) * A, t);
    const Vec<DIM> sp = lds_v<DIM>(raw + (2 * 2 + side) * A, t);
    const float is = raw[(3 * 2 + side) * A + t];
#pragma unroll
    for (int d = 0; d < DIM; ++d) out[0].c[d] = cg_u(r.c[d], w.c[d], sp.c[d], is, s.alpha[d], s.beta[d]);
  } else {
    const Vec<DIM> zw = lds_v<DIM>(raw + (0 * 2 + side) * A, t);
    Vec<DIM> z;
#pragma unroll
    for (int d = 0; d < DIM; ++d) z.c[d] = zw.c[d] - s.z0[d];
    out[0] = z;
    if constexpr (NC == 2) {
      const Vec<DIM> x = lds_v<DIM>(raw + (1 * 2 + side) * A, t);
#pragma unroll
      for (int d = 0; d < DIM; ++d) out[1].c[d] = sor_xt(z.c[d], x.c[d], s.om);
    }
  }
}

// --------------------------------------------------------------------------
// Row-block reduction of the partial buffers: thread t gets row R*TILE + t.
// --------------------------------------------------------------------------

// Row-block phase work unit: a quarter (32 rows) of row block R.  The four
// warps of the CTA take every fourth partial sum of the block's fixed list,
// for all 32 rows (lane = row), and the four part sums are added in warp
// order; warp 0 then holds the totals and runs the per-row epilogue.
constexpr int QROWS = 32;

// Sums the partials of rows R*TILE + 32*qr + lane and leaves the totals in
// shared memory, out[(c * QROWS + lane) * DIM + d] (valid for warp 0's use).
// Out of line with plain pointer arguments, so that its loads in flight get
// their own registers.
template <int DIM, int NC>
__device__ __noinline__ void reduce_quarter_smem(const float* __restrict__ part_i, const float* __restrict__ part_j,
                                                 const int* __restrict__ contrib_ptr,
                                                 const int* __restrict__ contrib, int R, int qr, int* idx,
                                                 float* scratch, float* out) {
  constexpr int DP = DimP<DIM>::v;
  constexpr int Q = 8;  // partials in flight per thread
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = QROWS * qr + lane;  // row inside the tile block
  Vec<DIM> s[NC], cmp[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    s[c] = vzero<DIM>();
    cmp[c] = vzero<DIM>();
  }
  const int c0 = contrib_ptr[R], c1 = contrib_ptr[R + 1];
  for (int base = c0; base < c1; base += CTA) {
    const int cnt = min(CTA, c1 - base);
    __syncthreads();
    if ((int)threadIdx.x < cnt) idx[threadIdx.x] = contrib[base + threadIdx.x];
    __syncthreads();
    for (int q0 = w; q0 < cnt; q0 += 4 * Q) {
      Vec<DIM> v[Q][NC];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = q0 + 4 * q;
        if (k < cnt) {
          const int e = idx[k];
          const float* src = (e >= 0) ? part_i + (size_t)e * 2 * TILE * DP : part_j + (size_t)(-1 - e) * 2 * TILE * DP;
#pragma unroll
          for (int c = 0; c < NC; ++c) v[q][c] = ldv<DIM>(src + (size_t)c * TILE * DP, row);
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q0 + 4 * q < cnt) {
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int d = 0; d < DIM; ++d) kahan_add(s[c].c[d], cmp[c].c[d], v[q][c].c[d]);
        }
    }
  }
  // part sums of the four warps, added in warp order
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int d = 0; d < DIM; ++d) scratch[((w * NC + c) * QROWS + lane) * DIM + d] = s[c].c[d] - cmp[c].c[d];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        float t = scratch[((0 * NC + c) * QROWS + lane) * DIM + d];
#pragma unroll
        for (int ww = 1; ww < 4; ++ww) t += scratch[((ww * NC + c) * QROWS + lane) * DIM + d];
        out[(c * QROWS + lane) * DIM + d] = t;
      }
  }
  __syncthreads();
}

template <int DIM, int NC>
__device__ __forceinline__ void reduce_rows(const KParams& p, int R, int qr, Vec<DIM> (&out)[NC]) {
  extern __shared__ __align__(256) unsigned char smem_dyn[];
  int* idx = reinterpret_cast<int*>(smem_dyn + SMEM_OFF_IDX);
  float* scratch = reinterpret_cast<float*>(smem_dyn + SMEM_OFF_POSI);      // free outside the passes
  float* res = scratch + 4 * 2 * QROWS * 3;
  reduce_quarter_smem<DIM, NC>(p.part_i, p.part_j, p.g.contrib_ptr, p.g.contrib, R, qr, idx, scratch, res);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int d = 0; d < DIM; ++d) out[c].c[d] = res[(c * QROWS + lane) * DIM + d];
}

// Warp-level double-float sum (fixed order); the totals land in lane 0.
template <int K>
__device__ __forceinline__ void warp_sum_df(df (&v)[K]) {
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
}

__device__ __forceinline__ float2* scal(const KParams& p, int parity) {
  return p.sc + (size_t)parity * 4 * p.g.nb * SC_STRIDE;
}

// Thread 0 of a CTA: bulk copies (TMA) of a tile's distance codes and of
// blocks I and J of every raw source array, completing on mbarrier b.
template <int DIM, int CODE, int SK>
__device__ __forceinline__ void issue_tile(const KParams& p, const PassSrc& src, unsigned char* smem, int tile, int I,
                                        int J, int b) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  constexpr unsigned TBYTES = TILE * TILE * CodeBytes<CODE>::v;
  constexpr int NA = SrcN<SK>::v;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
  float* raw = reinterpret_cast<float*>(smem + L::OFF_RAW);
  unsigned char* dbuf = smem + (b ? L::OFF_D1 : L::OFF_D0);
  unsigned bytes = TBYTES;
#pragma unroll
  for (int a = 0; a < NA; ++a) bytes += 2u * ((SK == SK_CGU && a == 3) ? TILE * 4 : TILE * DP * 4);
  fence_proxy_async();  // this CTA's reads of the raw area come before the copy overwrites it
  mbar_expect_tx(&mbar[b], bytes);
  bulk_g2s(dbuf, reinterpret_cast<const unsigned char*>(p.D) + (size_t)tile * TBYTES, TBYTES, &mbar[b]);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const bool scalar = (SK == SK_CGU && a == 3);
    const unsigned ab = scalar ? TILE * 4 : TILE * DP * 4;
    const int stride = scalar ? TILE : TILE * DP;
    bulk_g2s(raw + (a * 2 + 0) * TILE * DP, src.a[a] + (size_t)I * stride, ab, &mbar[b]);
    bulk_g2s(raw + (a * 2 + 1) * TILE * DP, src.a[a] + (size_t)J * stride, ab, &mbar[b]);
  }
}

// --------------------------------------------------------------------------
// A full pair pass: CTA b takes tasks b, b + G, b + 2G, ... (G = grid size);
// no global synchronisation inside the pass.
// --------------------------------------------------------------------------

template <int DIM, int MODE, int NC, int CODE, int SK>
__device__ bool pair_pass(const KParams& p, unsigned char* smem, PairState& ps, const PassSrc& src) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  const Geometry& g = p.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
  float* raw = reinterpret_cast<float*>(smem + L::OFF_RAW);
  float* posi = reinterpret_cast<float*>(smem + L::OFF_POSI);
  float* posj = reinterpret_cast<float*>(smem + L::OFF_POSJ);
  float2* red64 = reinterpret_cast<float2*>(smem + L::OFF_RED64);
  const unsigned char* lut = smem + L::OFF_LUT;
  float ssum[NC], scomp[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) ssum[c] = scomp[c] = 0.f;
  // vectors written before the last grid barrier are read below by bulk copies
  if (tid == 0) fence_proxy_async_global();
  int cur = blockIdx.x;
  if (cur < g.ntasks) {
    TaskDesc td = g.tasks[cur];
    int k = td.k0;
    int buf = 0;
    if (tid == 0) issue_tile<DIM, CODE, SK>(p, src, smem, td.tile0, td.I, (td.I + k) % g.nb, 0);
    Vec<DIM> iacc[NC][ROWS_PER_LANE];
    bool task_start = true;
    while (true) {
      const int J = (td.I + k) % g.nb;
      const int tile = td.tile0 + (k - td.k0);
      const unsigned ph = (ps.parity >> buf) & 1u;
      if (!mbar_wait(mbar + buf, ph, p.timeout_ns)) {
        set_error(p.ctrl, E_TIMEOUT);
        mbar_wait(mbar + buf, ph, p.timeout_ns);  // let our own copies land (bounded)
        return false;
      }
      ps.parity ^= (1u << buf);
      {
        Vec<DIM> vi[NC], vj[NC];
        form<DIM, SK, NC>(src, raw, 0, tid, vi);
        form<DIM, SK, NC>(src, raw, 1, tid, vj);
        // rows of block I are stored lane-interleaved: row 4l + a at a * 32 + l
        const int irow = (tid & (ROWS_PER_LANE - 1)) * 32 + (tid >> 2);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          sts_v<DIM>(posi + c * TILE * DP, irow, vi[c]);
          sts_v<DIM>(posj + c * TILE * DP, tid, vj[c]);
        }
      }
      __syncthreads();  // raw consumed; posi / posj ready
      const bool task_end = (k + 1 >= td.k1);
      int ntask = cur, nk = k + 1;
      TaskDesc ntd = td;
      if (task_end) {
        ntask = cur + gridDim.x;
        if (ntask < g.ntasks) {
          ntd = g.tasks[ntask];
          nk = ntd.k0;
        }
      }
      const bool more = ntask < g.ntasks;
      if (more && tid == 0)
        issue_tile<DIM, CODE, SK>(p, src, smem, ntd.tile0 + (nk - ntd.k0), ntd.I, (ntd.I + nk) % g.nb, buf ^ 1);

      if (task_start) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int a = 0; a < ROWS_PER_LANE; ++a) iacc[c][a] = vzero<DIM>();
        task_start = false;
      }
      Vec<DIM> xi[NC][ROWS_PER_LANE];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int a = 0; a < ROWS_PER_LANE; ++a) xi[c][a] = lds_v<DIM>(posi + c * TILE * DP, a * 32 + lane);
      Vec<DIM> jacc[NC];
      float st[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        st[c] = 0.f;
        jacc[c] = vzero<DIM>();
      }
      tile_compute<DIM, MODE, NC, CODE>(smem + (buf ? L::OFF_D1 : L::OFF_D0), posj, lut, xi, iacc, jacc, st, lane, warp);
#pragma unroll
      for (int c = 0; c < NC; ++c) kahan_add(ssum[c], scomp[c], st[c]);
      if constexpr (MODE != PM_STRESS) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          stv<DIM>(p.part_j + ((size_t)tile * 2 + c) * TILE * DP, warp * 32 + lane, jacc[c]);
      }
      if (task_end) {
        if constexpr (MODE != PM_STRESS) {
          __syncthreads();  // every warp is done with this distance buffer: reuse it for the row partials
          float* red = reinterpret_cast<float*>(smem + (buf ? L::OFF_D1 : L::OFF_D0));  // [4][NC][TILE][DP]
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int a = 0; a < ROWS_PER_LANE; ++a)
              sts_v<DIM>(red + ((size_t)(warp * NC + c) * TILE) * DP, ROWS_PER_LANE * lane + a, iacc[c][a]);
          __syncthreads();
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            Vec<DIM> s = lds_v<DIM>(red + ((size_t)(0 * NC + c) * TILE) * DP, tid);
#pragma unroll
            for (int w = 1; w < 4; ++w) {
              const Vec<DIM> v = lds_v<DIM>(red + ((size_t)(w * NC + c) * TILE) * DP, tid);
#pragma unroll
              for (int d = 0; d < DIM; ++d) s.c[d] += v.c[d];
            }
            stv<DIM>(p.part_i + ((size_t)cur * 2 + c) * TILE * DP, tid, s);
          }
        }
        task_start = true;
      }
      __syncthreads();
      if (!more) break;
      cur = ntask;
      td = ntd;
      k = nk;
      buf ^= 1;
    }
  }
  // stress of this CTA's pairs (candidates 0 and 1), one FP64 slot per CTA
  if constexpr (MODE == PM_STRESS || MODE == PM_RHS) {
    df v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = df_add(df_of(ssum[c]), df_of(-scomp[c]));
    cta_sum_multi<NC>(v, red64);
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) df_st(p.sc_cta + (size_t)blockIdx.x * 2 + c, v[c]);
    }
  }
  ps.pass += 1;
  return true;
}

// Runs an epilogue on every quarter row block (32 rows), one CTA per unit, after a pass.
template <class Epi>
__device__ __forceinline__ void rowblock_phase(const KParams& p, Epi& epi, int parity, float2* red64) {
  for (int u = blockIdx.x; u < 4 * p.g.nb; u += gridDim.x) epi(u >> 2, u & 3, parity, red64);
}

// --------------------------------------------------------------------------
// Epilogues (run once per row block, one CTA per block, after a pass)
// --------------------------------------------------------------------------

// Every epilogue below works on the 32 rows R*TILE + 32*qr + lane: the
// reduction uses the whole CTA, the per-row work runs in warp 0, and scalar
// partials go to slot (4*R + qr) of the row-block scalar array.

// b = L^{X} X of the initial layout (right-hand side of Eq. (2-5)).
template <int DIM>
struct EpiRhs0 {
  const KParams& p;
  __device__ __forceinline__ void operator()(int R, int qr, int, float2*) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, qr, acc);
    if (threadIdx.x < 32) stv<DIM>(p.B, R * TILE + QROWS * qr + threadIdx.x, acc[0]);
  }
};

// F = (L^X - L^W) X written to the caller's [n][dim] array.
template <int DIM>
struct EpiForces {
  const KParams& p;
  __device__ __forceinline__ void operator()(int R, int qr, int, float2*) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, qr, acc);
    const int i = R * TILE + QROWS * qr + threadIdx.x;
    if (threadIdx.x < 32 && i < p.g.n) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = acc[0].c[d];
    }
  }
};

__device__ __forceinline__ float2* scal_slot(const KParams& p, int parity, int R, int qr) {
  return scal(p, parity) + (size_t)(4 * R + qr) * SC_STRIDE;
}

// Start of an H step (Eq. (2-5)): take the layout x0 chosen by the previous
// acceptance test (or X^0), r0 = b - L^W x0, u0 = M^-1 r0, clear p and s;
// displacement sums of x0 against the previous layout.
// Scalar slots: [0,D) r.u  [D,2D) r.r  [2D,3D) b.b  [3D,4D) sum dx  [4D,5D) sum dx^2
//               [5D,6D) sum x  [6D,7D) sum x^2
template <int DIM>
struct EpiInit {
  const KParams& p;
  const float* x0src;
  bool first, accept;
  __device__ __forceinline__ void operator()(int R, int qr, int parity, float2*) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, qr, acc);
    if (threadIdx.x >= 32) return;
    const int i = R * TILE + QROWS * qr + threadIdx.x;
    const bool real = i < p.g.n;
    const Vec<DIM> x0 = ldv<DIM>(x0src, i), xo = ldv<DIM>(p.X, i);
    const Vec<DIM> b = first ? ldv<DIM>(p.B, i) : (accept ? ldv<DIM>(p.Bt, i) : ldv<DIM>(p.Bz, i));
    const float s = __ldcg(p.s + i), is = __ldcg(p.inv_s + i);
    Vec<DIM> r, u;
    df v[7 * DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      r.c[d] = b.c[d] - fmaf(s, x0.c[d], acc[0].c[d]);
      u.c[d] = is * r.c[d];
      const df dx = real ? df_diff(x0.c[d], xo.c[d]) : df_of(0.f);
      const float xv = real ? x0.c[d] : 0.f;
      v[d] = df_prod(r.c[d], u.c[d]);
      v[DIM + d] = df_prod(r.c[d], r.c[d]);
      v[2 * DIM + d] = df_prod(b.c[d], b.c[d]);
      v[3 * DIM + d] = dx;
      v[4 * DIM + d] = df_sqr(dx);
      v[5 * DIM + d] = df_of(xv);
      v[6 * DIM + d] = df_prod(xv, xv);
    }
    stv<DIM>(p.Zw, i, x0);
    stv<DIM>(p.X, i, x0);
    stv<DIM>(p.B, i, b);
    stv<DIM>(p.R, i, r);
    stv<DIM>(p.U, i, u);
    stv<DIM>(p.P, i, vzero<DIM>());
    stv<DIM>(p.S, i, vzero<DIM>());
    warp_sum_df<7 * DIM>(v);
    if (threadIdx.x == 0) {
      float2* o = scal_slot(p, parity, R, qr);
#pragma unroll
      for (int k = 0; k < 7 * DIM; ++k) df_st(o + k, v[k]);
    }
  }
};

// w0 = L^W u0 and delta0 = (w0, u0).  Slots [0,D).
template <int DIM>
struct EpiAU0 {
  const KParams& p;
  __device__ __forceinline__ void operator()(int R, int qr, int parity, float2*) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, qr, acc);
    if (threadIdx.x >= 32) return;
    const int i = R * TILE + QROWS * qr + threadIdx.x;
    const float s = __ldcg(p.s + i);
    const Vec<DIM> u = ldv<DIM>(p.U, i);
    Vec<DIM> w;
    df v[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      w.c[d] = fmaf(s, u.c[d], acc[0].c[d]);
      v[d] = df_prod(w.c[d], u.c[d]);
    }
    stv<DIM>(p.W, i, w);
    warp_sum_df<DIM>(v);
    if (threadIdx.x == 0) {
      float2* o = scal_slot(p, parity, R, qr);
#pragma unroll
      for (int k = 0; k < DIM; ++k) df_st(o + k, v[k]);
    }
  }
};

// One step of preconditioned CG in the single-reduction form of Chronopoulos
// and Gear: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s,
// u = M^-1 r, w = L^W u.  The curvature (p', L^W p') of the next direction
// p' = u + beta' p is needed before beta' is known; it is expanded as
// (u,w) + beta' ((u,s) + (p,w)) + beta'^2 (p,s) from dot products taken here,
// instead of the usual recurrence, which loses positivity in FP32.
// Slots: [0,D) r.u  [D,2D) w.u  [2D,3D) r.r  [3D,4D) u.s  [4D,5D) p.w  [5D,6D) p.s
template <int DIM>
struct EpiCG {
  const KParams& p;
  float alpha[3], beta[3];
  __device__ __forceinline__ void operator()(int R, int qr, int parity, float2*) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, qr, acc);
    if (threadIdx.x >= 32) return;
    const int i = R * TILE + QROWS * qr + threadIdx.x;
    const float s = __ldcg(p.s + i), is = __ldcg(p.inv_s + i);
    Vec<DIM> u = ldv<DIM>(p.U, i), w = ldv<DIM>(p.W, i), pp = ldv<DIM>(p.P, i), sp = ldv<DIM>(p.S, i);
    Vec<DIM> x = ldv<DIM>(p.Zw, i), r = ldv<DIM>(p.R, i);
    df v[6 * DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const float pn = fmaf(beta[d], pp.c[d], u.c[d]);
      const float sn = fmaf(beta[d], sp.c[d], w.c[d]);
      const float un = cg_u(r.c[d], w.c[d], sp.c[d], is, alpha[d], beta[d]);
      x.c[d] = fmaf(alpha[d], pn, x.c[d]);
      r.c[d] = fmaf(-alpha[d], sn, r.c[d]);
      pp.c[d] = pn;
      sp.c[d] = sn;
      u.c[d] = un;
      w.c[d] = fmaf(s, un, acc[0].c[d]);
      v[d] = df_prod(r.c[d], un);
      v[DIM + d] = df_prod(w.c[d], un);
      v[2 * DIM + d] = df_prod(r.c[d], r.c[d]);
      v[3 * DIM + d] = df_prod(un, sn);
      v[4 * DIM + d] = df_prod(pn, w.c[d]);
      v[5 * DIM + d] = df_prod(pn, sn);
    }
    stv<DIM>(p.P, i, pp);
    stv<DIM>(p.S, i, sp);
    stv<DIM>(p.Zw, i, x);
    stv<DIM>(p.R, i, r);
    stv<DIM>(p.U, i, u);
    stv<DIM>(p.W, i, w);
    warp_sum_df<6 * DIM>(v);
    if (threadIdx.x == 0) {
      float2* o = scal_slot(p, parity, R, qr);
#pragma unroll
      for (int k = 0; k < 6 * DIM; ++k) df_st(o + k, v[k]);
    }
  }
};

// After the stress/RHS pass of the two candidates: store X^{k+1} (pinned),
// the extrapolation X~ of Eq. (10) and both right-hand sides.
template <int DIM, int NC>
struct EpiK2 {
  const KParams& p;
  float z0[3];
  float om;
  __device__ __forceinline__ void operator()(int R, int qr, int, float2*) {
    Vec<DIM> acc[NC];
    reduce_rows<DIM, NC>(p, R, qr, acc);
    if (threadIdx.x >= 32) return;
    const int i = R * TILE + QROWS * qr + threadIdx.x;
    const bool real = i < p.g.n;
    const Vec<DIM> zw = ldv<DIM>(p.Zw, i), x = ldv<DIM>(p.X, i);
    Vec<DIM> z, xt;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      z.c[d] = real ? zw.c[d] - z0[d] : 0.f;
      xt.c[d] = real ? sor_xt(z.c[d], x.c[d], om) : 0.f;
    }
    stv<DIM>(p.Z, i, z);
    stv<DIM>(p.Xt, i, xt);
    stv<DIM>(p.Bz, i, acc[0]);
    stv<DIM>(p.Bt, i, acc[NC - 1]);
  }
};

// --------------------------------------------------------------------------
// The kernel
// --------------------------------------------------------------------------

__device__ __forceinline__ PassSrc direct_src(const float* a) {
  PassSrc s;
  s.a[0] = a;
  s.a[1] = s.a[2] = s.a[3] = nullptr;
#pragma unroll
  for (int d = 0; d < 3; ++d) s.alpha[d] = s.beta[d] = s.z0[d] = 0.f;
  s.om = 0.f;
  return s;
}

template <int DIM, int CODE>
__global__ void __launch_bounds__(CTA, (DIM == 3) ? 2 : 3) fd_main_kernel(KParams p) {
  using L = SmemLayout<DIM, CODE>;
  extern __shared__ __align__(256) unsigned char smem[];
  const Geometry& g = p.g;
  const int n = g.n, nb = g.nb, tid = threadIdx.x;
  float2* red64 = reinterpret_cast<float2*>(smem + L::OFF_RED64);
  Ctrl* ctrl = p.ctrl;

  // --- set-up: mbarriers and the replicated lookup table
  {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
    if (tid == 0) {
      mbar_init(&mbar[0], 1);
      mbar_init(&mbar[1], 1);
      fence_mbar_init();
    }
    if constexpr (CODE == CODE_U8) {
      uint4* dst = reinterpret_cast<uint4*>(smem + L::OFF_LUT);
      const uint4* srcl = reinterpret_cast<const uint4*>(p.lut);
      for (int k = tid; k < p.lut_rows * 16; k += CTA) dst[k] = srcl[k];
    }
    __syncthreads();
  }
  PairState ps;
  ps.parity = 0u;
  ps.pass = 0;
  int nbar = 0;
  if (p.timeline && blockIdx.x == 0 && tid == 0) ctrl->t_start = globaltimer_ns();
  auto mark = [&](int tag) {
    if (p.timeline && blockIdx.x == 0 && tid == 0 && ctrl->timeline_n < p.timeline_cap) {
      const int q = ctrl->timeline_n++;
      p.timeline[2 * q] = (double)tag;
      p.timeline[2 * q + 1] = (double)(globaltimer_ns() - ctrl->t_start);
    }
  };
  auto no_reduction = [] {};
  // grid barrier; the last CTA to arrive runs `red` first (a fixed-order reduction)
#define FD_SYNC_RED(tag, red)                                                   \
  do {                                                                          \
    if (!grid_sync_reduce(ctrl, p.timeout_ns, ++nbar, red)) return;             \
    mark(tag);                                                                  \
  } while (0)
#define FD_SYNC(tag) FD_SYNC_RED(tag, no_reduction)
  // reductions run by the last CTA
  auto red_stress = [&](int nc) {
    return [&, nc] {
      if (nc == 2) reduce_slots_to_ctrl<2>(ctrl, p.sc_cta, gridDim.x, 2, red64);
      else reduce_slots_to_ctrl<1>(ctrl, p.sc_cta, gridDim.x, 2, red64);
    };
  };

  // --- pack the caller layout into the padded internal array, check it
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
    stv<DIM>(p.X, i, v);
  }
  FD_SYNC(1);

  if (p.mode == KM_ENERGY) {
    if (!pair_pass<DIM, PM_STRESS, 1, CODE, SK_DIRECT>(p, smem, ps, direct_src(p.X))) return;
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
    EpiForces<DIM> e{p};
    if (!pair_pass<DIM, PM_FORCES, 1, CODE, SK_DIRECT>(p, smem, ps, direct_src(p.X))) return;
    FD_SYNC(3);
    rowblock_phase(p, e, 0, red64);
    if (blockIdx.x == 0 && tid == 0) {
      ctrl->pair_passes = 1.0;
      ctrl->stress_passes = 1.0;
    }
    return;
  }

  // ======================= KM_RUN: Algorithm 2 ============================
  // b = L^{X^0} X^0 and f(X^0) (right-hand side of Eq. (2-5), Eq. (1))
  if (!pair_pass<DIM, PM_RHS, 1, CODE, SK_DIRECT>(p, smem, ps, direct_src(p.X))) return;
  FD_SYNC_RED(4, red_stress(1));
  {
    EpiRhs0<DIM> e{p};
    rowblock_phase(p, e, 0, red64);
  }
  double f_cur;
  {
    df f[1];
    load_red<1>(ctrl, f);
    f_cur = df_to_double(f[0]);
  }
  if (!isfinite(f_cur)) {
    set_error(ctrl, E_NONFINITE);
    return;
  }
  if (blockIdx.x == 0 && tid == 0) p.trace_f[0] = f_cur;

  double passes_mv = 0.0, passes_st = 1.0;
  int cg_total = 0, cg_maxed = 0, cg_stalled = 0, n_acc = 0;
  double crit = 0.0;
  bool accept = true;
  double f_new = f_cur;
  int it_outer = 0;
  const float cgt2 = (float)(p.cg_tol * p.cg_tol);
  const int nunits = 4 * nb;
  for (int k = 0;; ++k) {
    // ---- start of the H step; also applies lines 6-8 of the previous iteration
    float rz[DIM], rr[DIM], bb[DIM];
    {
      const float* x0src = (k == 0) ? p.X : (accept ? p.Xt : p.Z);
      EpiInit<DIM> e{p, x0src, k == 0, accept};
      const int par = ps.pass & 1;
      if (!pair_pass<DIM, PM_MATVEC, 1, CODE, SK_DIRECT>(p, smem, ps, direct_src(x0src))) return;
      passes_mv += 1.0;
      FD_SYNC(5);
      rowblock_phase(p, e, par, red64);
      // reduce the 7*DIM sums; the last CTA also evaluates the termination rule
      const double fcur_k = f_cur, fnew_k = f_new;
      auto red_init = [&] {
        reduce_slots_to_ctrl<7 * DIM>(ctrl, scal(p, par), nunits, SC_STRIDE, red64);
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
      df v[3 * DIM];
      load_red<3 * DIM>(ctrl, v);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        rz[d] = df_f(v[d]);
        rr[d] = df_f(v[DIM + d]);
        bb[d] = df_f(v[2 * DIM + d]);
      }
      if (k > 0) {
        crit = __ldcg(&ctrl->red_d[0]);
        if (blockIdx.x == 0 && tid == 0) p.trace_crit[k - 1] = crit;
        f_cur = f_new;
        it_outer = k;
        if (crit < p.tol || k >= p.max_iter) break;
      }
    }
    // ---- CG on L^W Z = b, one reduction per step
    bool conv[DIM];
    bool all = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      conv[d] = (rr[d] <= cgt2 * bb[d]);
      all = all && conv[d];
    }
    int it = 0;
    if (!all) {
      float alpha[DIM], beta[DIM], gam[DIM];
      {
        EpiAU0<DIM> e{p};
        const int par = ps.pass & 1;
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE, SK_DIRECT>(p, smem, ps, direct_src(p.U))) return;
        passes_mv += 1.0;
        FD_SYNC(6);
        rowblock_phase(p, e, par, red64);
        auto red_au0 = [&] { reduce_slots_to_ctrl<DIM>(ctrl, scal(p, par), nunits, SC_STRIDE, red64); };
        FD_SYNC_RED(9, red_au0);
        df dlv[DIM];
        load_red<DIM>(ctrl, dlv);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float dl = df_f(dlv[d]);
          gam[d] = rz[d];
          beta[d] = 0.f;
          if (!conv[d] && !(dl > 0.f)) {
            conv[d] = true;  // u0 carries no curvature: nothing to solve in this column
            ++cg_stalled;
          }
          alpha[d] = conv[d] ? 0.f : gam[d] / dl;
        }
      }
      while (true) {
        PassSrc src = direct_src(p.R);
        src.a[1] = p.W;
        src.a[2] = p.S;
        src.a[3] = p.inv_s;
        EpiCG<DIM> e{p, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          src.alpha[d] = e.alpha[d] = alpha[d];
          src.beta[d] = e.beta[d] = beta[d];
        }
        const int par = ps.pass & 1;
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE, SK_CGU>(p, smem, ps, src)) return;
        passes_mv += 1.0;
        ++it;
        FD_SYNC(7);
        rowblock_phase(p, e, par, red64);
        auto red_cg = [&] { reduce_slots_to_ctrl<6 * DIM>(ctrl, scal(p, par), nunits, SC_STRIDE, red64); };
        FD_SYNC_RED(9, red_cg);
        df v[6 * DIM];
        load_red<6 * DIM>(ctrl, v);
        bool done = true;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float gn = df_f(v[d]), dn = df_f(v[DIM + d]), rrn = df_f(v[2 * DIM + d]);
          if (!conv[d]) {
            conv[d] = (rrn <= cgt2 * bb[d]);
            if (!conv[d]) {
              const float bn = gn / gam[d];
              const float pi = dn + bn * (df_f(v[3 * DIM + d]) + df_f(v[4 * DIM + d])) + bn * bn * df_f(v[5 * DIM + d]);
              if (pi > 0.f && gn > 0.f) {
                beta[d] = bn;
                alpha[d] = gn / pi;
              } else {
                conv[d] = true;  // curvature lost to rounding: the solve has gone as far as FP32 allows
                ++cg_stalled;
              }
            }
            if (conv[d]) {
              alpha[d] = 0.f;
              beta[d] = 0.f;
            }
          }
          gam[d] = gn;
          done = done && conv[d];
        }
        if (done) break;
        if (it >= p.cg_max) {
          ++cg_maxed;
          break;
        }
      }
    }
    cg_total += it;

    // ---- pin vertex 0 (Sec. 2), extrapolate (Eq. (10)), stress and RHS of both
    const double om = p.omega_seq[k];
    const bool two = (om != 0.0);
    PassSrc src = direct_src(p.Zw);
    src.a[1] = p.X;
    {
      const Vec<DIM> z0 = ldv<DIM>(p.Zw, 0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) src.z0[d] = z0.c[d];
      src.om = (float)om;
    }
    if (two) {
      EpiK2<DIM, 2> e{p, {src.z0[0], src.z0[1], src.z0[2]}, src.om};
      if (!pair_pass<DIM, PM_RHS, 2, CODE, SK_K2>(p, smem, ps, src)) return;
      passes_st += 2.0;
      FD_SYNC_RED(8, red_stress(2));
      rowblock_phase(p, e, 0, red64);
    } else {
      EpiK2<DIM, 1> e{p, {src.z0[0], src.z0[1], src.z0[2]}, src.om};
      if (!pair_pass<DIM, PM_RHS, 1, CODE, SK_K2>(p, smem, ps, src)) return;
      passes_st += 1.0;
      FD_SYNC_RED(8, red_stress(1));
      rowblock_phase(p, e, 0, red64);
    }
    df fz[2];
    load_red<2>(ctrl, fz);
    FD_SYNC(9);  // Z, X~ and their right-hand sides are complete
    const double fZ = df_to_double(fz[0]);
    const double fT = two ? df_to_double(fz[1]) : fZ;
    if (!isfinite(fZ) || !isfinite(fT)) {
      set_error(ctrl, E_NONFINITE);
      return;
    }
    // line 6 (ties accept).  With omega = 0 the two candidates coincide and
    // X^{k+1} is kept as it is (the test is trivially true).
    accept = two && (fT <= fZ);
    f_new = accept ? fT : fZ;
    if (accept || !two) ++n_acc;
    if (blockIdx.x == 0 && tid == 0) {
      p.trace_f[k + 1] = f_new;
      p.trace_acc[k] = (accept || !two) ? 1 : 0;
      p.trace_om[k] = om;
      p.trace_cg[k] = it;
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
    ctrl->iters = it_outer;
    ctrl->cg_steps = cg_total;
    ctrl->cg_maxed = cg_maxed;
    ctrl->cg_stalled = cg_stalled;
    ctrl->accepted = n_acc;
    ctrl->f_final = f_cur;
    ctrl->crit_final = crit;
    ctrl->pair_passes = passes_mv + passes_st;
    ctrl->matvec_passes = passes_mv;
    ctrl->stress_passes = passes_st;
  }
#undef FD_SYNC
#undef FD_SYNC_RED
}

}  // namespace fdl
