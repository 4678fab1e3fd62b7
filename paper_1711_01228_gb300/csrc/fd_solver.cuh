// fd_solver.cuh -- the cooperative layout kernel (stress, forces, and the
// whole Algorithm 2 loop of Wang & Wang 2012) for one layout dimension and
// one distance-code type.  Included by fd_solver_d{1,2,3}.cu.
//
// Work decomposition
// ------------------
// All-pairs passes run over the tiles of the half-ring (fd_internal.cuh),
// grouped into tasks of consecutive tiles of one block row.  CTAs take tasks
// from a global ticket counter.  A CTA has 4 warps; every warp holds all 128
// rows of block I (4 rows per lane, in registers) and sweeps 32 columns of
// block J.  In step t lane l pairs its 4 rows with column 32w + ((l + t) & 31);
// the column accumulators travel one lane down after every step, so after 32
// steps each lane holds the complete column sums of its own column and both
// endpoints of every pair are accumulated exactly once (symmetric n-body).
// Distance codes of a tile (16 KB for uint8) are staged in shared memory by a
// 1-D bulk copy (TMA) that is prefetched one tile ahead; column positions are
// staged by the CTA's threads.
//
// Per-tile column partials and per-task row partials go to global buffers and
// are summed per row block in a fixed order (Kahan-compensated), so results
// do not depend on which CTA ran which task.  Scalars (stress, CG dot
// products, displacement sums) are reduced in FP64 in a fixed order.
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

// shared-memory vector access (plain loads/stores)
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

// A source of per-vertex vectors for a pair pass: a + beta * b (b optional).
template <int DIM>
struct Src {
  const float* a;
  const float* b;
  float beta[DIM];
  __device__ __forceinline__ Vec<DIM> load(int i) const {
    Vec<DIM> v = ldv<DIM>(a, i);
    if (b != nullptr) {
      Vec<DIM> w = ldv<DIM>(b, i);
#pragma unroll
      for (int d = 0; d < DIM; ++d) v.c[d] = fmaf(beta[d], w.c[d], v.c[d]);
    }
    return v;
  }
};

template <int DIM>
__device__ __forceinline__ Src<DIM> make_src(const float* a) {
  Src<DIM> s;
  s.a = a;
  s.b = nullptr;
#pragma unroll
  for (int d = 0; d < DIM; ++d) s.beta[d] = 0.f;
  return s;
}

enum PairMode { PM_STRESS = 0, PM_FORCES = 1, PM_RHS = 2, PM_MATVEC = 3 };

template <int CODE>
struct CodeBytes {
  static constexpr int v = (CODE == CODE_U8) ? 1 : 4;
};

// Shared memory of the kernel.  The column partial "red" area aliases the
// distance buffer that has just been consumed.
template <int DIM, int CODE>
struct SmemLayout {
  static constexpr int DP = DimP<DIM>::v;
  static constexpr int DBUF = TILE * TILE * CodeBytes<CODE>::v;
  static constexpr int OFF_D0 = 0;
  static constexpr int OFF_D1 = DBUF;
  static constexpr int OFF_POS = 2 * DBUF;                      // [2][TILE][DP] floats
  static constexpr int OFF_LUT2 = OFF_POS + 2 * TILE * DP * 4;  // float2 [LUT_N] {1/d, -1}
  static constexpr int OFF_LUTF = OFF_LUT2 + LUT_N * 8;         // float2 [LUT_N] {1/d, 1/d^2}
  static constexpr int OFF_LUTW = OFF_LUTF + LUT_N * 8;         // float  [LUT_N] 1/d^2
  static constexpr int OFF_RED64 = OFF_LUTW + LUT_N * 4;        // double [CTA]
  static constexpr int OFF_MISC = OFF_RED64 + CTA * 8;          // mbar[2], task slots
  static constexpr int BYTES = OFF_MISC + 64;
  static_assert(4 * 2 * TILE * DP * 4 <= DBUF, "row partial area must fit in a distance buffer");
};

struct PairState {
  unsigned long long ticket_base;
  unsigned parity[2];
};

// --------------------------------------------------------------------------
// Deterministic FP64 reductions across a CTA
// --------------------------------------------------------------------------

// Sum of v over the CTA's threads, fixed tree order; result valid in all threads.
__device__ __forceinline__ double cta_sum_f64(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = CTA / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// Sum over a strided FP64 array a[i * stride + off], i < count; every CTA
// obtains the identical value.
__device__ __forceinline__ double sum_strided_f64(const double* a, int count, int stride, int off,
                                                  double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += CTA) v += __ldcg(a + (size_t)i * stride + off);
  return cta_sum_f64(v, red);
}

// --------------------------------------------------------------------------
// One tile of a pair pass
// --------------------------------------------------------------------------

template <int DIM, int MODE, int NC, int CODE>
__device__ __forceinline__ void tile_compute(const unsigned char* __restrict__ dt, const float* __restrict__ posj,
                                             const float2* __restrict__ lut2, const float2* __restrict__ lutf,
                                             const float* __restrict__ lutw, const Vec<DIM> (&xi)[NC][ROWS_PER_LANE],
                                             Vec<DIM> (&iacc)[NC][ROWS_PER_LANE], Vec<DIM> (&jacc)[NC],
                                             float (&st)[NC], int lane, int warp) {
  constexpr int DP = DimP<DIM>::v;
  constexpr float TINY = 1e-30f;  // keeps rsqrt finite for coincident points; below FP32 resolution of r^2
#pragma unroll 1
  for (int t = 0; t < 32; ++t) {
    const int jl = warp * 32 + ((lane + t) & 31);
    float dv[ROWS_PER_LANE];
    unsigned codes = 0;
    if constexpr (CODE == CODE_U8) {
      codes = *reinterpret_cast<const unsigned*>(dt + jl * TILE + ROWS_PER_LANE * lane);
    } else {
      float4 q = *reinterpret_cast<const float4*>(dt + 4 * (jl * TILE + ROWS_PER_LANE * lane));
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
      float invd, negm, w;
      if constexpr (CODE == CODE_U8) {
        const unsigned code = (codes >> (8 * a)) & 0xFFu;
        if constexpr (MODE == PM_MATVEC) {
          w = lutw[code];
          invd = 0.f;
          negm = 0.f;
        } else if constexpr (MODE == PM_FORCES) {
          float2 l = lutf[code];
          invd = l.x;
          w = l.y;
          negm = 0.f;
        } else {
          float2 l = lut2[code];
          invd = l.x;
          negm = l.y;
          w = 0.f;
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
          jacc[0].c[d] = fmaf(-w, xi[0][a].c[d], jacc[0].c[d]);
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
              jacc[c].c[d] = fmaf(-coef, dx[d], jacc[c].c[d]);
            }
          }
        }
      }
    }
    if constexpr (MODE != PM_STRESS) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int d = 0; d < DIM; ++d) jacc[c].c[d] = __shfl_sync(0xffffffffu, jacc[c].c[d], (lane + 1) & 31);
    }
  }
}

// --------------------------------------------------------------------------
// A full pair pass over all tasks (dynamic scheduling)
// --------------------------------------------------------------------------

template <int DIM, int CODE>
__device__ __forceinline__ const unsigned char* tile_ptr(const KParams& p, int tile) {
  return reinterpret_cast<const unsigned char*>(p.D) + (size_t)tile * (TILE * TILE * CodeBytes<CODE>::v);
}

template <int DIM, int MODE, int NC, int CODE>
__device__ bool pair_pass(const KParams& p, unsigned char* smem, PairState& ps, const Src<DIM> (&src)[NC]) {
  using L = SmemLayout<DIM, CODE>;
  constexpr int DP = DimP<DIM>::v;
  constexpr unsigned TBYTES = TILE * TILE * CodeBytes<CODE>::v;
  const Geometry& g = p.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
  int* slot = reinterpret_cast<int*>(smem + L::OFF_MISC + 16);
  float* posj = reinterpret_cast<float*>(smem + L::OFF_POS);
  const float2* lut2 = reinterpret_cast<const float2*>(smem + L::OFF_LUT2);
  const float2* lutf = reinterpret_cast<const float2*>(smem + L::OFF_LUTF);
  const float* lutw = reinterpret_cast<const float*>(smem + L::OFF_LUTW);
  double* red64 = reinterpret_cast<double*>(smem + L::OFF_RED64);
  unsigned char* dbuf[2] = {smem + L::OFF_D0, smem + L::OFF_D1};

  auto grab = [&]() -> int {
    if (threadIdx.x == 0) {
      unsigned long long t = atomicAdd(&p.ctrl->ticket, 1ull) - ps.ticket_base;
      slot[0] = (t < (unsigned long long)g.ntasks) ? (int)t : -1;
    }
    __syncthreads();
    int r = slot[0];
    __syncthreads();
    return r;
  };

  bool ok = true;
  int cur = grab();
  int buf = 0;
  if (cur >= 0) {
    TaskDesc td = g.tasks[cur];
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(&mbar[0], TBYTES);
      bulk_g2s(dbuf[0], tile_ptr<DIM, CODE>(p, td.tile0), TBYTES, &mbar[0]);
    }
    int k = td.k0;
    Vec<DIM> xi[NC][ROWS_PER_LANE];
    Vec<DIM> iacc[NC][ROWS_PER_LANE];
    float ssum[NC], scomp[NC];
    while (true) {
      if (k == td.k0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
          for (int a = 0; a < ROWS_PER_LANE; ++a) {
            xi[c][a] = src[c].load(td.I * TILE + ROWS_PER_LANE * lane + a);
#pragma unroll
            for (int d = 0; d < DIM; ++d) iacc[c][a].c[d] = 0.f;
          }
          ssum[c] = 0.f;
          scomp[c] = 0.f;
        }
      }
      const int J = (td.I + k) % g.nb;
      const int tile = td.tile0 + (k - td.k0);
      // next tile (same task, or the first tile of a new task)
      int ntask = cur, nk = k + 1;
      TaskDesc ntd = td;
      if (nk >= td.k1) {
        ntask = grab();
        if (ntask >= 0) {
          ntd = g.tasks[ntask];
          nk = ntd.k0;
        }
      }
      if (ntask >= 0 && threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(&mbar[buf ^ 1], TBYTES);
        bulk_g2s(dbuf[buf ^ 1], tile_ptr<DIM, CODE>(p, ntd.tile0 + (nk - ntd.k0)), TBYTES, &mbar[buf ^ 1]);
      }
      // column vectors of block J
#pragma unroll
      for (int c = 0; c < NC; ++c)
        for (int jj = threadIdx.x; jj < TILE; jj += CTA) sts_v<DIM>(posj + c * TILE * DP, jj, src[c].load(J * TILE + jj));
      __syncthreads();
      if (!mbar_wait(&mbar[buf], ps.parity[buf], p.timeout_ns)) {
        set_error(p.ctrl, E_TIMEOUT);
        // let our own copies land before leaving (bounded)
        mbar_wait(&mbar[buf], ps.parity[buf], p.timeout_ns);
        if (ntask >= 0) mbar_wait(&mbar[buf ^ 1], ps.parity[buf ^ 1], p.timeout_ns);
        return false;
      }
      ps.parity[buf] ^= 1u;

      Vec<DIM> jacc[NC];
      float st[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        st[c] = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) jacc[c].c[d] = 0.f;
      }
      tile_compute<DIM, MODE, NC, CODE>(dbuf[buf], posj, lut2, lutf, lutw, xi, iacc, jacc, st, lane, warp);
      if constexpr (MODE != PM_STRESS) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          stv<DIM>(p.part_j + ((size_t)tile * 2 + c) * TILE * DP, warp * 32 + lane, jacc[c]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) kahan_add(ssum[c], scomp[c], st[c]);
      __syncthreads();  // dbuf[buf] and posj are free again

      if (nk >= td.k1 || ntask != cur) {
        // task finished: row partials summed over the 4 warps in fixed order
        if constexpr (MODE != PM_STRESS) {
          float* red = reinterpret_cast<float*>(dbuf[buf]);  // [4][NC][TILE][DP]
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int a = 0; a < ROWS_PER_LANE; ++a)
              sts_v<DIM>(red + ((size_t)(warp * NC + c) * TILE) * DP, ROWS_PER_LANE * lane + a, iacc[c][a]);
          __syncthreads();
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int row = threadIdx.x;  // CTA == TILE
            Vec<DIM> s = lds_v<DIM>(red + ((size_t)(0 * NC + c) * TILE) * DP, row);
#pragma unroll
            for (int w = 1; w < 4; ++w) {
              Vec<DIM> v = lds_v<DIM>(red + ((size_t)(w * NC + c) * TILE) * DP, row);
#pragma unroll
              for (int d = 0; d < DIM; ++d) s.c[d] += v.c[d];
            }
            stv<DIM>(p.part_i + ((size_t)cur * 2 + c) * TILE * DP, row, s);
          }
        }
        if constexpr (MODE == PM_STRESS || MODE == PM_RHS) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            double tot = cta_sum_f64((double)ssum[c] - (double)scomp[c], red64);
            if (threadIdx.x == 0) __stcg(p.sc_task + (size_t)cur * 2 + c, tot);
          }
        }
        __syncthreads();
      }
      if (ntask < 0) break;
      if (ntask != cur) {
        cur = ntask;
        td = ntd;
      }
      k = nk;
      buf ^= 1;
    }
  }
  ps.ticket_base += (unsigned long long)g.ntasks + gridDim.x;
  return ok;
}

// --------------------------------------------------------------------------
// Row-block reduction of the partial buffers: thread t gets row R*TILE + t.
// --------------------------------------------------------------------------

template <int DIM, int NC>
__device__ __forceinline__ void reduce_rows(const KParams& p, int R, Vec<DIM> (&out)[NC]) {
  constexpr int DP = DimP<DIM>::v;
  const Geometry& g = p.g;
  const int row = threadIdx.x;
  Vec<DIM> s[NC], cmp[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      s[c].c[d] = 0.f;
      cmp[c].c[d] = 0.f;
    }
  const int t0 = g.strip_task_base[R], t1 = g.strip_task_base[R + 1];
  for (int t = t0; t < t1; ++t) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Vec<DIM> v = ldv<DIM>(p.part_i + ((size_t)t * 2 + c) * TILE * DP, row);
#pragma unroll
      for (int d = 0; d < DIM; ++d) kahan_add(s[c].c[d], cmp[c].c[d], v.c[d]);
    }
  }
  for (int I = 0; I < g.nb; ++I) {
    int k = R - I;
    if (k < 0) k += g.nb;
    if (k >= g.strip_len[I]) continue;
    const int tile = g.tile_base[I] + k;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Vec<DIM> v = ldv<DIM>(p.part_j + ((size_t)tile * 2 + c) * TILE * DP, row);
#pragma unroll
      for (int d = 0; d < DIM; ++d) kahan_add(s[c].c[d], cmp[c].c[d], v.c[d]);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int d = 0; d < DIM; ++d) out[c].c[d] = s[c].c[d] - cmp[c].c[d];
}

// --------------------------------------------------------------------------
// The kernel
// --------------------------------------------------------------------------

template <int DIM, int CODE>
__global__ void __launch_bounds__(CTA) fd_main_kernel(KParams p) {
  using L = SmemLayout<DIM, CODE>;
  extern __shared__ __align__(128) unsigned char smem[];
  const Geometry& g = p.g;
  const int n = g.n, nb = g.nb, tid = threadIdx.x;
  double* red64 = reinterpret_cast<double*>(smem + L::OFF_RED64);

  // --- set-up: mbarriers and lookup tables in shared memory
  {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_MISC);
    if (tid == 0) {
      mbar_init(&mbar[0], 1);
      mbar_init(&mbar[1], 1);
      fence_mbar_init();
    }
    float2* lut2 = reinterpret_cast<float2*>(smem + L::OFF_LUT2);
    float2* lutf = reinterpret_cast<float2*>(smem + L::OFF_LUTF);
    float* lutw = reinterpret_cast<float*>(smem + L::OFF_LUTW);
    for (int i = tid; i < LUT_N; i += CTA) {
      float4 e = p.lut[i];
      lut2[i] = make_float2(e.x, e.z);
      lutf[i] = make_float2(e.x, e.y);
      lutw[i] = e.y;
    }
    __syncthreads();
  }
  PairState ps;
  ps.ticket_base = 0;
  ps.parity[0] = ps.parity[1] = 0;
  int nbar = 0;
#define FD_SYNC()                                              \
  do {                                                         \
    if (!grid_sync(p.ctrl, p.timeout_ns, ++nbar)) return;      \
  } while (0)

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
    if (bad) set_error(p.ctrl, E_NONFINITE);
    stv<DIM>(p.X, i, v);
  }
  FD_SYNC();

  if (p.mode == KM_ENERGY) {
    Src<DIM> s1[1] = {make_src<DIM>(p.X)};
    if (!pair_pass<DIM, PM_STRESS, 1, CODE>(p, smem, ps, s1)) return;
    FD_SYNC();
    if (blockIdx.x == 0) {
      double f = sum_strided_f64(p.sc_task, g.ntasks, 2, 0, red64);
      if (tid == 0) {
        p.ctrl->f_final = f;
        p.ctrl->pair_passes += 1.0;
        p.ctrl->stress_passes += 1.0;
        if (!isfinite(f)) set_error(p.ctrl, E_NONFINITE);
      }
    }
    return;
  }

  if (p.mode == KM_FORCES) {
    Src<DIM> s1[1] = {make_src<DIM>(p.X)};
    if (!pair_pass<DIM, PM_FORCES, 1, CODE>(p, smem, ps, s1)) return;
    FD_SYNC();
    for (int R = blockIdx.x; R < nb; R += gridDim.x) {
      Vec<DIM> acc[1];
      reduce_rows<DIM, 1>(p, R, acc);
      const int i = R * TILE + tid;
      if (i < n) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = acc[0].c[d];
      }
    }
    if (blockIdx.x == 0 && tid == 0) {
      p.ctrl->pair_passes += 1.0;
      p.ctrl->stress_passes += 1.0;
    }
    return;
  }

  // ======================= KM_RUN: Algorithm 2 ============================
  // b = L^{X^0} X^0 and f(X^0) (Eq. (2-5) right-hand side, Eq. (1))
  {
    Src<DIM> s1[1] = {make_src<DIM>(p.X)};
    if (!pair_pass<DIM, PM_RHS, 1, CODE>(p, smem, ps, s1)) return;
  }
  FD_SYNC();
  double f_cur = sum_strided_f64(p.sc_task, g.ntasks, 2, 0, red64);
  if (!isfinite(f_cur)) {
    set_error(p.ctrl, E_NONFINITE);
    return;
  }
  for (int R = blockIdx.x; R < nb; R += gridDim.x) {
    Vec<DIM> acc[1];
    reduce_rows<DIM, 1>(p, R, acc);
    const int i = R * TILE + tid;
    stv<DIM>(p.B, i, acc[0]);
    stv<DIM>(p.Zw, i, ldv<DIM>(p.X, i));  // warm start of the first solve
  }
  if (blockIdx.x == 0 && tid == 0) {
    p.trace_f[0] = f_cur;
    p.ctrl->pair_passes += 1.0;
    p.ctrl->stress_passes += 1.0;
  }
  FD_SYNC();

  int cg_total = 0, cg_maxed = 0, n_acc = 0;
  double crit = 0.0;
  int it_outer = 0;
  for (; it_outer < p.max_iter;) {
    // ---------------- H step: CG on L^W Z = b (Eq. (2-5)) ----------------
    {
      Src<DIM> s1[1] = {make_src<DIM>(p.Zw)};
      if (!pair_pass<DIM, PM_MATVEC, 1, CODE>(p, smem, ps, s1)) return;
    }
    FD_SYNC();
    // r = b - L^W z, zc = r / s, p = zc
    for (int R = blockIdx.x; R < nb; R += gridDim.x) {
      Vec<DIM> acc[1];
      reduce_rows<DIM, 1>(p, R, acc);
      const int i = R * TILE + tid;
      const float s = __ldcg(p.s + i), is = __ldcg(p.inv_s + i);
      Vec<DIM> z = ldv<DIM>(p.Zw, i), b = ldv<DIM>(p.B, i), r, zc;
      double prz[DIM], prr[DIM], pbb[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const float q = fmaf(s, z.c[d], acc[0].c[d]);
        r.c[d] = b.c[d] - q;
        zc.c[d] = r.c[d] * is;
        prz[d] = (double)r.c[d] * (double)zc.c[d];
        prr[d] = (double)r.c[d] * (double)r.c[d];
        pbb[d] = (double)b.c[d] * (double)b.c[d];
      }
      stv<DIM>(p.R, i, r);
      stv<DIM>(p.Zc, i, zc);
      stv<DIM>(p.Pa, i, zc);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double a1 = cta_sum_f64(prz[d], red64);
        double a2 = cta_sum_f64(prr[d], red64);
        double a3 = cta_sum_f64(pbb[d], red64);
        if (tid == 0) {
          p.sc_a[R * 8 + d] = a1;
          p.sc_a[R * 8 + 3 + d] = a2;
          p.sc_b[R * 8 + d] = a3;
        }
      }
    }
    if (blockIdx.x == 0 && tid == 0) {
      p.ctrl->pair_passes += 1.0;
      p.ctrl->matvec_passes += 1.0;
    }
    FD_SYNC();
    double rz[DIM], bb[DIM], beta[DIM];
    bool conv[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      rz[d] = sum_strided_f64(p.sc_a, nb, 8, d, red64);
      const double rr = sum_strided_f64(p.sc_a, nb, 8, 3 + d, red64);
      bb[d] = sum_strided_f64(p.sc_b, nb, 8, d, red64);
      conv[d] = (rr <= p.cg_tol * p.cg_tol * bb[d]);
      beta[d] = 0.0;
    }
    float* pold = p.Pa;
    float* pnew = p.Pb;
    int it = 0;
    while (true) {
      bool all = true;
#pragma unroll
      for (int d = 0; d < DIM; ++d) all = all && conv[d];
      if (all) break;
      if (it >= p.cg_max) {
        ++cg_maxed;
        break;
      }
      // q = L^W p with p = zc + beta * p_old formed on the fly
      {
        Src<DIM> s1[1];
        s1[0].a = p.Zc;
        s1[0].b = pold;
#pragma unroll
        for (int d = 0; d < DIM; ++d) s1[0].beta[d] = (float)beta[d];
        if (!pair_pass<DIM, PM_MATVEC, 1, CODE>(p, smem, ps, s1)) return;
      }
      FD_SYNC();
      for (int R = blockIdx.x; R < nb; R += gridDim.x) {
        Vec<DIM> acc[1];
        reduce_rows<DIM, 1>(p, R, acc);
        const int i = R * TILE + tid;
        const float s = __ldcg(p.s + i);
        Vec<DIM> zc = ldv<DIM>(p.Zc, i), po = ldv<DIM>(pold, i), pn, q;
        double ppq[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          pn.c[d] = fmaf((float)beta[d], po.c[d], zc.c[d]);
          q.c[d] = fmaf(s, pn.c[d], acc[0].c[d]);
          ppq[d] = (double)pn.c[d] * (double)q.c[d];
        }
        stv<DIM>(pnew, i, pn);
        stv<DIM>(p.Q, i, q);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          double a = cta_sum_f64(ppq[d], red64);
          if (tid == 0) p.sc_b[R * 8 + 3 + d] = a;
        }
      }
      if (blockIdx.x == 0 && tid == 0) {
      p.ctrl->pair_passes += 1.0;
      p.ctrl->matvec_passes += 1.0;
    }
      FD_SYNC();
      double alpha[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double pq = sum_strided_f64(p.sc_b, nb, 8, 3 + d, red64);
        if (conv[d]) {
          alpha[d] = 0.0;
        } else if (!(pq > 0.0)) {
          set_error(p.ctrl, E_CG_BREAKDOWN);
          return;
        } else {
          alpha[d] = rz[d] / pq;
        }
      }
      for (int R = blockIdx.x; R < nb; R += gridDim.x) {
        const int i = R * TILE + tid;
        const float is = __ldcg(p.inv_s + i);
        Vec<DIM> z = ldv<DIM>(p.Zw, i), r = ldv<DIM>(p.R, i), pn = ldv<DIM>(pnew, i), q = ldv<DIM>(p.Q, i), zc;
        double prz[DIM], prr[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float a = (float)alpha[d];
          z.c[d] = fmaf(a, pn.c[d], z.c[d]);
          r.c[d] = fmaf(-a, q.c[d], r.c[d]);
          zc.c[d] = r.c[d] * is;
          prz[d] = (double)r.c[d] * (double)zc.c[d];
          prr[d] = (double)r.c[d] * (double)r.c[d];
        }
        stv<DIM>(p.Zw, i, z);
        stv<DIM>(p.R, i, r);
        stv<DIM>(p.Zc, i, zc);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          double a1 = cta_sum_f64(prz[d], red64);
          double a2 = cta_sum_f64(prr[d], red64);
          if (tid == 0) {
            p.sc_a[R * 8 + d] = a1;
            p.sc_a[R * 8 + 3 + d] = a2;
          }
        }
      }
      FD_SYNC();
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double rzn = sum_strided_f64(p.sc_a, nb, 8, d, red64);
        const double rr = sum_strided_f64(p.sc_a, nb, 8, 3 + d, red64);
        if (!conv[d]) {
          beta[d] = (rz[d] != 0.0) ? rzn / rz[d] : 0.0;
          conv[d] = (rr <= p.cg_tol * p.cg_tol * bb[d]);
        } else {
          beta[d] = 0.0;
        }
        rz[d] = rzn;
      }
      float* t = pold;
      pold = pnew;
      pnew = t;
      ++it;
    }
    cg_total += it;

    // ------------- pin vertex 0 (Sec. 2) and extrapolate (Eq. (10)) -------------
    const double om = p.omega_seq[it_outer];
    const float omf = (float)om;
    {
      const Vec<DIM> z0 = ldv<DIM>(p.Zw, 0);
      for (int R = blockIdx.x; R < nb; R += gridDim.x) {
        const int i = R * TILE + tid;
        Vec<DIM> z = ldv<DIM>(p.Zw, i), x = ldv<DIM>(p.X, i), zz, xt;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          zz.c[d] = (i < n) ? z.c[d] - z0.c[d] : 0.f;
          xt.c[d] = (i < n) ? fmaf(1.0f + omf, zz.c[d], -omf * x.c[d]) : 0.f;
        }
        stv<DIM>(p.Z, i, zz);
        stv<DIM>(p.Xt, i, xt);
      }
    }
    FD_SYNC();

    // ------------- stress and RHS of both candidates (Algorithm 2 lines 4-6) ----
    const bool two = (om != 0.0);
    if (two) {
      Src<DIM> s2[2] = {make_src<DIM>(p.Z), make_src<DIM>(p.Xt)};
      if (!pair_pass<DIM, PM_RHS, 2, CODE>(p, smem, ps, s2)) return;
    } else {
      Src<DIM> s1[1] = {make_src<DIM>(p.Z)};
      if (!pair_pass<DIM, PM_RHS, 1, CODE>(p, smem, ps, s1)) return;
    }
    FD_SYNC();
    const double fZ = sum_strided_f64(p.sc_task, g.ntasks, 2, 0, red64);
    const double fT = two ? sum_strided_f64(p.sc_task, g.ntasks, 2, 1, red64) : fZ;
    if (!isfinite(fZ) || !isfinite(fT)) {
      set_error(p.ctrl, E_NONFINITE);
      return;
    }
    const bool accept = (fT <= fZ);  // line 6; ties accept
    const double f_new = accept ? fT : fZ;
    // lines 7-8: keep the chosen layout and its RHS; displacement sums
    for (int R = blockIdx.x; R < nb; R += gridDim.x) {
      const int i = R * TILE + tid;
      Vec<DIM> acc[2];
      if (two) {
        reduce_rows<DIM, 2>(p, R, acc);
      } else {
        Vec<DIM> a1[1];
        reduce_rows<DIM, 1>(p, R, a1);
        acc[0] = a1[0];
        acc[1] = a1[0];
      }
      Vec<DIM> xo = ldv<DIM>(p.X, i);
      Vec<DIM> xn = (accept && two) ? ldv<DIM>(p.Xt, i) : ldv<DIM>(p.Z, i);
      const Vec<DIM>& bn = (accept && two) ? acc[1] : acc[0];
      double sd[DIM], sd2[DIM], sx[DIM], sx2[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double dlt = (i < n) ? (double)xn.c[d] - (double)xo.c[d] : 0.0;
        const double xv = (i < n) ? (double)xn.c[d] : 0.0;
        sd[d] = dlt;
        sd2[d] = dlt * dlt;
        sx[d] = xv;
        sx2[d] = xv * xv;
      }
      stv<DIM>(p.X, i, xn);
      stv<DIM>(p.B, i, bn);
      stv<DIM>(p.Zw, i, xn);  // warm start of the next solve
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double a1 = cta_sum_f64(sd[d], red64);
        double a2 = cta_sum_f64(sd2[d], red64);
        double a3 = cta_sum_f64(sx[d], red64);
        double a4 = cta_sum_f64(sx2[d], red64);
        if (tid == 0) {
          p.sc_a[R * 8 + d] = a1;
          p.sc_a[R * 8 + 3 + d] = a2;
          p.sc_b[R * 8 + d] = a3;
          p.sc_b[R * 8 + 3 + d] = a4;
        }
      }
    }
    FD_SYNC();
    // termination criterion (same value in every CTA)
    if (p.stop == 0) {
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double s1 = sum_strided_f64(p.sc_a, nb, 8, d, red64);
        const double s2 = sum_strided_f64(p.sc_a, nb, 8, 3 + d, red64);
        const double x1 = sum_strided_f64(p.sc_b, nb, 8, d, red64);
        const double x2 = sum_strided_f64(p.sc_b, nb, 8, 3 + d, red64);
        num += fmax(s2 - s1 * s1 / n, 0.0);
        den += fmax(x2 - x1 * x1 / n, 0.0);
      }
      crit = (den > 0.0) ? sqrt(num / den) : 0.0;
    } else {
      crit = (f_cur != 0.0) ? (f_cur - f_new) / f_cur : 0.0;
    }
    if (accept && two) ++n_acc;
    else if (!two) ++n_acc;
    if (blockIdx.x == 0 && tid == 0) {
      p.trace_f[it_outer + 1] = f_new;
      p.trace_acc[it_outer] = accept ? 1 : 0;
      p.trace_om[it_outer] = om;
      p.trace_cg[it_outer] = it;
      p.trace_crit[it_outer] = crit;
      p.ctrl->pair_passes += two ? 2.0 : 1.0;
      p.ctrl->stress_passes += two ? 2.0 : 1.0;
    }
    f_cur = f_new;
    ++it_outer;
    if (crit < p.tol) break;
  }

  // --- output
  for (int R = blockIdx.x; R < nb; R += gridDim.x) {
    const int i = R * TILE + tid;
    if (i < n) {
      Vec<DIM> x = ldv<DIM>(p.X, i);
#pragma unroll
      for (int d = 0; d < DIM; ++d) p.x_out[(size_t)i * DIM + d] = x.c[d];
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    p.ctrl->iters = it_outer;
    p.ctrl->cg_steps = cg_total;
    p.ctrl->cg_maxed = cg_maxed;
    p.ctrl->accepted = n_acc;
    p.ctrl->f_final = f_cur;
    p.ctrl->crit_final = crit;
  }
#undef FD_SYNC
}

}  // namespace fdl
