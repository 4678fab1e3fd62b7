// fd_batch.cuh -- many independent small layouts in one persistent launch.
//
// Each CTA takes whole graphs from a queue (largest first) and runs the
// complete Algorithm 2 of Wang & Wang 2012 for one graph at a time: right-hand
// side and stress (Prop. 2.1, Eq. (1)), the H step by preconditioned CG on
// Eq. (2-5) with the first vertex pinned, the extrapolation of Eq. (10), the
// acceptance test of line 6 and the termination rule.  No grid-wide
// synchronisation: graphs never share a CTA, so a CTA barrier is the only
// barrier, and a CTA's reductions stay in shared memory.
//
// Tile edge per graph.  A graph's pairs are cut into T x T tiles with
// T = 32, 64 or 128 (its blocks of T vertices in the half-ring order of
// fd_internal.cuh), chosen per size bucket by the host's autotuner: small
// graphs waste most of a 128 x 128 tile on padding.  The CTA's W * 128
// threads form W * 128 / T tile groups of T threads, which split the tiles of
// a pass (contiguous ranges of the half ring).  A group runs the same
// symmetric tile arithmetic as the single-graph kernel (tile_compute in
// fd_solver.cuh at edge T), with the tile's distance codes arriving by 1-D
// bulk copies (TMA) into the group's own stages.  Every per-vertex vector of
// the graph lives in shared memory or in L2-resident pools: the pass input
// V[nb][NC][T][DP] and the pass sums A[NC][n_pad][DP] in shared memory
// (column and row sums are added with shared-memory atomics, because two
// groups may touch one block), the CG state in global pools.
//
// Graphs up to BMAX_N vertices with hop diameter up to 253 (uint8 codes).
#pragma once

#include "fd_solver.cuh"

namespace fdl {

constexpr int BGT = 128;          // threads of one 128-thread unit (a CTA has W = 1 or 2 units)
constexpr int BMAX_W = 2;         // 128-thread units per CTA
constexpr int BMAX_G = BMAX_W * BGT / 32;  // tile groups per CTA at the smallest tile (T = 32)
constexpr int BMAX_NBUF = 3;      // stages per group
// Stage bytes per 128 threads and stage: at tile edge T the 128 / T groups of
// T threads hold T * T bytes each, T * 128 <= TILE * TILE in all.
constexpr int BTILE_BYTES = TILE * TILE;

// Shared-memory layout of the batched kernel.
template <int DIM>
struct BSmem {
  static constexpr int DP = DimP<DIM>::v;
  static constexpr int OFF_RED = 0;       // double [warps][BRED_K] reduction scratch
  static constexpr int BRED_K = 8;
  static constexpr int OFF_MBAR = 1024;   // [BMAX_G][BMAX_NBUF] mbarriers
  static constexpr int OFF_ST = 1280;     // BState
  static constexpr int OFF_P = 2048;      // copy of BParams
  static constexpr int OFF_LUT = 3072;
  __host__ __device__ static constexpr int off_v(int lut_bytes) { return align_up(OFF_LUT + lut_bytes, 128); }
  __host__ __device__ static constexpr int v_bytes(int n_pad) { return 2 * n_pad * DP * 4; }
  __host__ __device__ static constexpr int off_a(int lut_bytes, int n_pad) { return off_v(lut_bytes) + v_bytes(n_pad); }
  __host__ __device__ static constexpr int off_stage(int lut_bytes, int n_pad) {
    return off_a(lut_bytes, n_pad) + v_bytes(n_pad);
  }
  __host__ __device__ static constexpr int bytes(int lut_bytes, int n_pad, int W, int nbuf) {
    return off_stage(lut_bytes, n_pad) + W * nbuf * BTILE_BYTES;
  }
};

// Per-graph scalars of the Algorithm 2 loop (shared memory).
struct BState {
  double f_cur, f_new, crit, pmv, pst;
  double red[16];        // results of the last CTA reduction
  float rz[3], bb[3], alpha[3], beta[3];
  int conv[3];
  int graph, it, cg_total, n_acc, stop, abort, status, k;
  unsigned parity;       // mbarrier phase bits of every group (bit w * BMAX_NBUF + s, w < BMAX_G)
  int pass;
};
static_assert(sizeof(BState) <= 2048 - 1280, "BState must fit its slot");
static_assert(BMAX_G * BMAX_NBUF * 8 <= 1280 - 1024 && BMAX_G * BMAX_NBUF <= 32, "mbarrier slots and parity bits");
static_assert(sizeof(BParams) <= 3072 - 2048, "BParams must fit its slot");

// Barrier of tile group w (T threads; named barrier 1 + w, barrier 0 is the CTA's).
template <int T>
__device__ __forceinline__ void group_sync(int w) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + w), "r"(T) : "memory");
}

// Group barrier that also ANDs a predicate over the group's threads.
template <int T>
__device__ __forceinline__ bool group_and(int w, bool pred) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(1 + w), "r"(T)
      : "memory");
  return r != 0;
}

// Sums K doubles over the CTA in a fixed order; thread 0 writes them to st->red.
template <int K>
__device__ __forceinline__ void bcta_sum(double (&v)[K], double* scratch, BState* st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += scratch[w * K + k];
      st->red[k] = t;
    }
  }
  __syncthreads();
}

// Index of candidate c of padded vertex i in the pass input V[nb][NC][T][DP]
// (blocks of the graph's tile edge T).
template <int DIM, int T>
__device__ __forceinline__ int vidx(int i, int c, int nc) {
  return (((i / T) * nc + c) * T + (i % T)) * DimP<DIM>::v;
}

__device__ __forceinline__ void s_red_add(float* a, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(a)), "f"(v) : "memory");
}

// --------------------------------------------------------------------------
// One all-pairs pass over the T x T tiles of one graph (T = 32, 64 or 128,
// chosen per graph).  The CTA's W * 128 threads form GW = W * 128 / T tile
// groups of T threads; group w takes tiles [T_g w / GW, T_g (w + 1) / GW) of
// the strip-major order (T_g tiles in all) from the codes at Dg.  Sums go to
// A (candidate c at A + c * n_pad_max * DP), stress per candidate to
// st->red[c].  Returns false (and sets st->abort) if a copy wait timed out.
// --------------------------------------------------------------------------
template <int DIM, int MODE, int NC, int W, int T>
__device__ __noinline__ bool bpass(int n, int nb, const unsigned char* Dg) {
  extern __shared__ __align__(256) unsigned char smem[];
  using SL = BSmem<DIM>;
  using TS = TileShape<DIM, MODE, T>;
  constexpr int R = TS::R, G = TS::G, DP = DimP<DIM>::v;
  constexpr int GW = W * BGT / T;      // tile groups of the CTA
  constexpr int TB = T * T;            // code bytes of one tile
  constexpr int NWG = (T + 31) / 32;   // warps of a group
  static_assert(GW <= BMAX_G, "mbarrier slots");
  const BParams& p = *reinterpret_cast<const BParams*>(smem + SL::OFF_P);
  BState* st = reinterpret_cast<BState*>(smem + SL::OFF_ST);
  const int lut_bytes = p.lut_rows * LUT_ROW;
  const unsigned char* lut = smem + SL::OFF_LUT;
  const float* V = reinterpret_cast<const float*>(smem + SL::off_v(lut_bytes));
  float* A = reinterpret_cast<float*>(smem + SL::off_a(lut_bytes, p.n_pad_max));
  unsigned char* stg0 = smem + SL::off_stage(lut_bytes, p.n_pad_max);
  uint64_t* mbar0 = reinterpret_cast<uint64_t*>(smem + SL::OFF_MBAR);
  const int w = threadIdx.x / T, tid = threadIdx.x % T, nbuf = p.nbuf;
  const int astride = p.n_pad_max * DP;
  const int NT = hr_tiles(nb);
  const int ta = (int)((long long)NT * w / GW), tb = (int)((long long)NT * (w + 1) / GW);
  unsigned char* stg = stg0 + (size_t)w * nbuf * TB;
  uint64_t* mbar = mbar0 + w * BMAX_NBUF;
  unsigned parity = (st->parity >> (w * BMAX_NBUF)) & ((1u << BMAX_NBUF) - 1u);
  constexpr int NS = NStress<MODE, NC>::v;
  float ssum[NS], scomp[NS];
#pragma unroll
  for (int c = 0; c < NS; ++c) ssum[c] = scomp[c] = 0.f;
  bool ok = true;
  unsigned inflight = 0u;  // stages with a copy issued by this thread and not yet consumed
  if (ta < tb) {
    // the first nbuf - 1 tiles of the range
    if (tid == 0) {
      for (int k = 0; k < nbuf - 1 && ta + k < tb; ++k) {
        fence_proxy_async();
        mbar_expect_tx(mbar + k, TB);
        bulk_g2s(stg + k * TB, Dg + (size_t)(ta + k) * TB, TB, mbar + k);
        inflight |= 1u << k;
      }
    }
    int I = 0;
    while (hr_base(nb, I + 1) <= ta) ++I;
    int k = ta - hr_base(nb, I);
    int LI = hr_len(nb, I);
    Rows<DIM, NC, R> rows;
    bool fresh = true;  // rows of block I not loaded yet
    int s = 0;
    for (int t = ta; t < tb; ++t) {
      const int J = (I + k) % nb;
      const unsigned ph = (parity >> s) & 1u;
      // the group decides together (a thread whose own wait timed out makes
      // every thread of the group leave); also the barrier after which the
      // stage of the previous tile may be refilled
      if (!group_and<T>(w, mbar_wait(mbar + s, ph, p.timeout_ns))) {
        ok = false;
        st->abort = 1;
        break;
      }
      parity ^= 1u << s;
      inflight &= ~(1u << s);
      if (tid == 0 && t + nbuf - 1 < tb) {
        const int sn = (s + nbuf - 1) % nbuf;
        fence_proxy_async();
        mbar_expect_tx(mbar + sn, TB);
        bulk_g2s(stg + sn * TB, Dg + (size_t)(t + nbuf - 1) * TB, TB, mbar + sn);
        inflight |= 1u << sn;
      }
      const int q = tid & (G - 1);
      if (fresh) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int a2 = 0; a2 < R / 2; ++a2) {
            const int i0 = I * T + R * q + 2 * a2;
            const Vec<DIM> x0 = lds_v<DIM>(V, vidx<DIM, T>(i0, c, NC) / DP);
            const Vec<DIM> x1 = lds_v<DIM>(V, vidx<DIM, T>(i0 + 1, c, NC) / DP);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              rows.x[c][d][a2] = pk2(x0.c[d], x1.c[d]);
              rows.acc[c][d][a2] = pk2(0.f, 0.f);
            }
          }
        fresh = false;
      }
      Vec<DIM> jout[NC];
      float stv_[NS];
      const unsigned char* dt = stg + s * TB;
      const float* colv = V + (size_t)J * NC * T * DP;
      const bool edge = (k == 0) || (n < nb * T && (I == nb - 1 || J == nb - 1));
      if (edge) tile_compute<DIM, MODE, NC, CODE_U8, true, T>(dt, colv, lut, rows, jout, stv_, tid);
      else tile_compute<DIM, MODE, NC, CODE_U8, false, T>(dt, colv, lut, rows, jout, stv_, tid);
      if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L) {
#pragma unroll
        for (int c = 0; c < NS; ++c) kahan_add(ssum[c], scomp[c], stv_[c]);
      }
      if constexpr (MODE != PM_STRESS) {
        const int j = J * T + tid;
        if (j < n) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (MODE == PM_K2L && c != NC - 1) continue;  // no right-hand side of the first candidate
#pragma unroll
            for (int d = 0; d < DIM; ++d)
              s_red_add(A + c * astride + j * DP + d, (MODE == PM_MATVEC) ? jout[c].c[d] : -jout[c].c[d]);
          }
        }
        // row sums when the range leaves block row I: the column groups of a
        // warp are added by shuffles, the group's warps meet in the stage's
        // code buffer ([NC][warps][T][DP] floats: NC * DP * T * T / 8 bytes)
        const bool last = (t + 1 == tb) || (k + 1 == LI);
        if (last) {
          float* red = reinterpret_cast<float*>(stg + s * TB);
          const int lane = tid & 31, wl = tid >> 5;
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
              for (int a2 = 0; a2 < R / 2; ++a2) {
                if (MODE == PM_K2L && c != NC - 1) continue;
                float lo = lo2(rows.acc[c][d][a2]), hi = hi2(rows.acc[c][d][a2]);
#pragma unroll
                for (int m = G; m < 32 && m < T; m <<= 1) {
                  lo += __shfl_xor_sync(0xffffffffu, lo, m);
                  hi += __shfl_xor_sync(0xffffffffu, hi, m);
                }
                rows.acc[c][d][a2] = pk2(lo, hi);
              }
          group_sync<T>(w);  // every thread is done with the codes
          if (lane < G) {
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
                float* base = red + ((size_t)(c * NWG + wl) * T) * DP;
                sts_v<DIM>(base, R * q + 2 * a2, v0);
                sts_v<DIM>(base, R * q + 2 * a2 + 1, v1);
              }
          }
          group_sync<T>(w);
          const int i = I * T + tid;
          if (i < n) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              if (MODE == PM_K2L && c != NC - 1) continue;
              Vec<DIM> sm = lds_v<DIM>(red + ((size_t)(c * NWG) * T) * DP, tid);
#pragma unroll
              for (int gg = 1; gg < NWG; ++gg) {
                const Vec<DIM> v = lds_v<DIM>(red + ((size_t)(c * NWG + gg) * T) * DP, tid);
#pragma unroll
                for (int d = 0; d < DIM; ++d) sm.c[d] += v.c[d];
              }
#pragma unroll
              for (int d = 0; d < DIM; ++d) s_red_add(A + c * astride + i * DP + d, sm.c[d]);
            }
          }
          fresh = true;
        }
      } else {
        if (k + 1 == LI) fresh = true;
      }
      if (++k == LI) {
        ++I;
        k = 0;
        LI = (I < nb) ? hr_len(nb, I) : 0;
      }
      s = (s + 1 == nbuf) ? 0 : s + 1;
    }
    if (!ok && tid == 0) {
      // let the copies this thread issued land (bounded) before the CTA leaves
      for (int b = 0; b < nbuf; ++b)
        if (inflight & (1u << b)) mbar_wait(mbar + b, (parity >> b) & 1u, p.timeout_ns);
    }
  }
  // publish this group's parity, then the CTA's stress sums
  __syncthreads();
  if (tid == 0) {
    atomicAnd(&st->parity, ~(((1u << BMAX_NBUF) - 1u) << (w * BMAX_NBUF)));
    atomicOr(&st->parity, parity << (w * BMAX_NBUF));
  }
  if constexpr (MODE == PM_STRESS || MODE == PM_RHS || MODE == PM_K2L) {
    double v[NS];
#pragma unroll
    for (int c = 0; c < NS; ++c) v[c] = (double)ssum[c] - (double)scomp[c];
    bcta_sum<NS>(v, reinterpret_cast<double*>(smem + SL::OFF_RED), st);
  } else {
    __syncthreads();
  }
  return !st->abort;
}

// --------------------------------------------------------------------------
// Algorithm 2 for one graph, by the whole CTA.
// --------------------------------------------------------------------------
template <int DIM, int W, int T>
__device__ __forceinline__ void run_graph(int g) {
  extern __shared__ __align__(256) unsigned char smem[];
  using SL = BSmem<DIM>;
  constexpr int DP = DimP<DIM>::v;
  const BParams& p = *reinterpret_cast<const BParams*>(smem + SL::OFF_P);
  BState* st = reinterpret_cast<BState*>(smem + SL::OFF_ST);
  double* scratch = reinterpret_cast<double*>(smem + SL::OFF_RED);
  const int lut_bytes = p.lut_rows * LUT_ROW;
  float* V = reinterpret_cast<float*>(smem + SL::off_v(lut_bytes));
  float* A0 = reinterpret_cast<float*>(smem + SL::off_a(lut_bytes, p.n_pad_max));
  float* A1 = A0 + p.n_pad_max * DP;
  const BGraph gr = p.graphs[g];
  // blocks of the graph's tile edge T (32, 64 or 128) and its codes
  constexpr int lgT = (T == 32) ? 5 : (T == 64) ? 6 : 7;
  const int n = gr.n, nb = gr.nbt, n_pad = nb * T;
  const unsigned char* Dg = (T == TILE) ? p.D + (size_t)gr.t0 * TILE * TILE : p.DT + gr.dt;
  const size_t vo = (size_t)gr.p0 * DP;
  float* X = p.X + vo;
  float* Z = p.Z + vo;
  float* Rr = p.R + vo;
  float* Pp = p.Pd + vo;
  float* B = p.B + vo;
  float* R0 = p.R0 + vo;
  const float* S = p.s + gr.p0;
  const float* IS = p.inv_s + gr.p0;
  const float* xin = p.x_in + (size_t)gr.v0 * DIM;
  float* xout = p.x_out + (size_t)gr.v0 * DIM;
  const int tid = threadIdx.x, nt = blockDim.x;
  const float cgt2 = (float)(p.cg_tol * p.cg_tol);
  const unsigned long long t_start = globaltimer_ns();

  // load X^0, clear the pass sums
  int bad = 0;
  for (int i = tid; i < n_pad; i += nt) {
    Vec<DIM> x;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const float v = (i < n) ? __ldcg(xin + (size_t)i * DIM + d) : 0.f;
      if (!isfinite(v)) bad = 1;
      x.c[d] = v;
    }
    stv<DIM>(X, i, x);
    sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, x);
  }
  for (int e = tid; e < 2 * p.n_pad_max * DP; e += nt) A0[e] = 0.f;
  if (tid == 0) {
    st->graph = g;
    st->abort = 0;
    st->status = 0;
    st->pmv = st->pst = 0.0;
    st->cg_total = st->n_acc = st->k = 0;
    st->crit = 0.0;
  }
  bad = __syncthreads_or(bad);
  auto finish = [&](int iters) {
    for (int i = tid; i < n; i += nt) {
      const Vec<DIM> x = ldv<DIM>(X, i);
#pragma unroll
      for (int d = 0; d < DIM; ++d) xout[(size_t)i * DIM + d] = x.c[d];
    }
    if (tid == 0) {
      p.iters[g] = iters;
      p.cg_steps[g] = st->cg_total;
      p.accepted[g] = st->n_acc;
      p.status[g] = st->status;
      p.f_final[g] = st->f_cur;
      p.crit_final[g] = st->crit;
      p.passes_mv[g] = st->pmv;
      p.passes_st[g] = st->pst;
      p.graph_ms[g] = (double)(globaltimer_ns() - t_start) * 1e-6;
    }
  };
  if (bad) {
    if (tid == 0) {
      st->status = E_NONFINITE;
      st->f_cur = 0.0;
    }
    __syncthreads();
    finish(0);
    return;
  }
  // b = L^{X^0} X^0 and f(X^0)
  if (!bpass<DIM, PM_RHS, 1, W, T>(n, nb, Dg)) return;
  if (tid == 0) {
    st->f_cur = st->red[0];
    st->pst += 1.0;
    if (!isfinite(st->f_cur)) st->status = E_NONFINITE;
  }
  for (int i = tid; i < n_pad; i += nt) {
    Vec<DIM> b;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      b.c[d] = A0[i * DP + d];
      A0[i * DP + d] = 0.f;
    }
    stv<DIM>(B, i, b);
  }
  __syncthreads();
  if (st->status != 0 || n == 1) {
    finish(0);
    return;
  }

  int k = 0;
  for (;; ++k) {
    // ---- H step: L^W Z = B by Jacobi-preconditioned CG from Z = X^k.  The
    // starting residual B - L^W X^k takes an all-pairs pass at the first
    // iteration and every LWX_REFRESH-th; in between the previous iteration
    // left it in R0 (L^W X^k from that H step's B, R and R0, as in the
    // single-graph kernel).
    const bool lwx_pass = (k % LWX_REFRESH) == 0;
    if (lwx_pass) {
      for (int i = tid; i < n_pad; i += nt) sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, ldv<DIM>(X, i));
      __syncthreads();
      if (!bpass<DIM, PM_MATVEC, 1, W, T>(n, nb, Dg)) return;
    }
    {
      double v[3 * DIM];
#pragma unroll
      for (int e = 0; e < 3 * DIM; ++e) v[e] = 0.0;
      for (int i = tid; i < n_pad; i += nt) {
        const Vec<DIM> x = ldv<DIM>(X, i), b = ldv<DIM>(B, i);
        const float s = __ldcg(S + i), is = __ldcg(IS + i);
        const Vec<DIM> r0 = lwx_pass ? vzero<DIM>() : ldv<DIM>(R0, i);
        Vec<DIM> r, u;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          if (lwx_pass) {
            const float a = A0[i * DP + d];
            A0[i * DP + d] = 0.f;
            r.c[d] = b.c[d] - fmaf(s, x.c[d], -a);
          } else {
            r.c[d] = r0.c[d];
          }
          u.c[d] = is * r.c[d];
          v[d] += (double)(r.c[d] * u.c[d]);
          v[DIM + d] += (double)(r.c[d] * r.c[d]);
          v[2 * DIM + d] += (double)(b.c[d] * b.c[d]);
        }
        stv<DIM>(Z, i, x);
        stv<DIM>(Rr, i, r);
        stv<DIM>(R0, i, r);
        stv<DIM>(Pp, i, u);
        sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, u);
      }
      if (tid == 0 && lwx_pass) st->pmv += 1.0;
      bcta_sum<3 * DIM>(v, scratch, st);
      if (tid == 0) {
        for (int d = 0; d < DIM; ++d) {
          st->rz[d] = (float)st->red[d];
          st->bb[d] = (float)st->red[2 * DIM + d];
          st->conv[d] = ((float)st->red[DIM + d] <= cgt2 * st->bb[d]) ? 1 : 0;
        }
        st->it = 0;
      }
      __syncthreads();
    }
    while (true) {
      bool all = true;
#pragma unroll
      for (int d = 0; d < DIM; ++d) all = all && st->conv[d];
      if (all) break;
      if (st->it >= p.cg_max) break;
      if (!bpass<DIM, PM_MATVEC, 1, W, T>(n, nb, Dg)) return;
      // q = L^W p (kept in A0), (p, q)
      {
        double v[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) v[d] = 0.0;
        for (int i = tid; i < n_pad; i += nt) {
          const Vec<DIM> pp = ldv<DIM>(Pp, i);
          const float s = __ldcg(S + i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const float q = fmaf(s, pp.c[d], -A0[i * DP + d]);
            A0[i * DP + d] = q;
            v[d] += (double)(pp.c[d] * q);
          }
        }
        if (tid == 0) {
          st->pmv += 1.0;
          ++st->it;
        }
        bcta_sum<DIM>(v, scratch, st);
        if (tid == 0) {
          for (int d = 0; d < DIM; ++d) {
            const float pq = (float)st->red[d];
            if (st->conv[d]) {
              st->alpha[d] = 0.f;
            } else if (!(pq > 0.f)) {
              st->alpha[d] = 0.f;  // no curvature left in FP32: the column stops here
              st->conv[d] = 1;
            } else {
              st->alpha[d] = st->rz[d] / pq;
            }
          }
        }
        __syncthreads();
      }
      // z += alpha p, r -= alpha q, u = M^-1 r
      {
        float al[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) al[d] = st->alpha[d];
        double v[2 * DIM];
#pragma unroll
        for (int e = 0; e < 2 * DIM; ++e) v[e] = 0.0;
        for (int i = tid; i < n_pad; i += nt) {
          Vec<DIM> z = ldv<DIM>(Z, i), r = ldv<DIM>(Rr, i);
          const Vec<DIM> pp = ldv<DIM>(Pp, i);
          const float is = __ldcg(IS + i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const float q = A0[i * DP + d];
            A0[i * DP + d] = 0.f;
            z.c[d] = fmaf(al[d], pp.c[d], z.c[d]);
            r.c[d] = fmaf(-al[d], q, r.c[d]);
            const float u = is * r.c[d];
            v[d] += (double)(r.c[d] * u);
            v[DIM + d] += (double)(r.c[d] * r.c[d]);
          }
          stv<DIM>(Z, i, z);
          stv<DIM>(Rr, i, r);
        }
        bcta_sum<2 * DIM>(v, scratch, st);
        if (tid == 0) {
          for (int d = 0; d < DIM; ++d) {
            const float rzn = (float)st->red[d], rr = (float)st->red[DIM + d];
            if (!st->conv[d]) {
              st->beta[d] = (st->rz[d] > 0.f) ? rzn / st->rz[d] : 0.f;
              st->rz[d] = rzn;
              if (rr <= cgt2 * st->bb[d]) st->conv[d] = 1;
            } else {
              st->beta[d] = 0.f;
            }
          }
        }
        __syncthreads();
      }
      // p = u + beta p
      {
        float be[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) be[d] = st->beta[d];
        for (int i = tid; i < n_pad; i += nt) {
          const Vec<DIM> r = ldv<DIM>(Rr, i);
          Vec<DIM> pp = ldv<DIM>(Pp, i);
          const float is = __ldcg(IS + i);
#pragma unroll
          for (int d = 0; d < DIM; ++d) pp.c[d] = fmaf(be[d], pp.c[d], is * r.c[d]);
          stv<DIM>(Pp, i, pp);
          sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, pp);
        }
        __syncthreads();
      }
    }
    // ---- pin vertex 0 (Sec. 2), extrapolate (Eq. (10)), stress and RHS of both candidates
    const double om_d = p.omega_seq ? p.omega_seq[k] : p.omega[g];
    const float om = (float)om_d;
    const bool two = (om_d != 0.0);
    const Vec<DIM> z0 = ldv<DIM>(Z, 0);
    __syncthreads();  // every thread has read z_0 before it is overwritten
    for (int i = tid; i < n_pad; i += nt) {
      const Vec<DIM> zw = ldv<DIM>(Z, i), x = ldv<DIM>(X, i);
      Vec<DIM> z, xt;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        z.c[d] = (i < n) ? zw.c[d] - z0.c[d] : 0.f;
        xt.c[d] = (i < n) ? sor_xt(z.c[d], x.c[d], om) : 0.f;
      }
      stv<DIM>(Z, i, z);
      if (two) {
        sts_v<DIM>(V, vidx<DIM, T>(i, 0, 2) / DP, z);
        sts_v<DIM>(V, vidx<DIM, T>(i, 1, 2) / DP, xt);
      } else {
        sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, z);
      }
    }
    if (tid == 0) st->cg_total += st->it;
    __syncthreads();
    // both candidates' stresses, the right-hand side of the extrapolated one
    // only (line 6 mostly keeps it); a pass for z's follows when z is kept
    if (two) {
      if (!bpass<DIM, PM_K2L, 2, W, T>(n, nb, Dg)) return;
    } else {
      if (!bpass<DIM, PM_RHS, 1, W, T>(n, nb, Dg)) return;
    }
    const double fZ = st->red[0], fT = two ? st->red[1] : st->red[0];
    const bool accept = two && (fT <= fZ);  // line 6, ties accept
    const double f_prev = st->f_cur, f_next = accept ? fT : fZ;
    if (two && !accept) {
      for (int i = tid; i < n_pad; i += nt) sts_v<DIM>(V, vidx<DIM, T>(i, 0, 1) / DP, ldv<DIM>(Z, i));
      __syncthreads();
      if (!bpass<DIM, PM_RHS, 1, W, T>(n, nb, Dg)) return;  // z's right-hand side into A0
      if (tid == 0) st->pst += 1.0;
    }
    // X^{k+1}, its right-hand side, and the displacement sums of the termination rule
    {
      double v[4 * DIM];
#pragma unroll
      for (int e = 0; e < 4 * DIM; ++e) v[e] = 0.0;
      for (int i = tid; i < n_pad; i += nt) {
        const Vec<DIM> z = ldv<DIM>(Z, i), x = ldv<DIM>(X, i);
        // this H step's B, final residual R = B - L^W z and starting residual
        // R0 = B - L^W X^k give L^W X^{k+1} (z or the extrapolation) and the
        // next step's starting residual without a pass
        const Vec<DIM> bo = ldv<DIM>(B, i), rf = ldv<DIM>(Rr, i), r0 = ldv<DIM>(R0, i);
        Vec<DIM> xn, b, r0n;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          xn.c[d] = accept ? ((i < n) ? sor_xt(z.c[d], x.c[d], om) : 0.f) : z.c[d];
          const float b0 = A0[i * DP + d], b1 = two ? A1[i * DP + d] : 0.f;
          A0[i * DP + d] = 0.f;
          if (two) A1[i * DP + d] = 0.f;
          b.c[d] = accept ? b1 : b0;
          const float lz = bo.c[d] - rf.c[d];
          const float lwx = accept ? fmaf(1.f + om, lz, -om * (bo.c[d] - r0.c[d])) : lz;
          r0n.c[d] = b.c[d] - lwx;
          if (i < n) {
            const double dx = (double)xn.c[d] - (double)x.c[d];
            v[d] += (double)xn.c[d];
            v[DIM + d] += (double)xn.c[d] * (double)xn.c[d];
            v[2 * DIM + d] += dx;
            v[3 * DIM + d] += dx * dx;
          }
        }
        stv<DIM>(X, i, xn);
        stv<DIM>(B, i, b);
        stv<DIM>(R0, i, r0n);
      }
      bcta_sum<4 * DIM>(v, scratch, st);
      if (tid == 0) {
        double c;
        if (p.stop == 0) {
          double num = 0.0, den = 0.0;
          for (int d = 0; d < DIM; ++d) {
            num += fmax(st->red[3 * DIM + d] - st->red[2 * DIM + d] * st->red[2 * DIM + d] / n, 0.0);
            den += fmax(st->red[DIM + d] - st->red[d] * st->red[d] / n, 0.0);
          }
          c = (den > 0.0) ? sqrt(num / den) : 0.0;
        } else {
          c = (f_prev != 0.0) ? (f_prev - f_next) / f_prev : 0.0;
        }
        st->crit = c;
        st->f_cur = f_next;
        st->pst += two ? 2.0 : 1.0;
        if (accept || !two) ++st->n_acc;
        if (!isfinite(f_next)) st->status = E_NONFINITE;
        st->stop = (st->status != 0 || c < p.tol || k + 1 >= p.max_iter) ? 1 : 0;
      }
      __syncthreads();
    }
    if (st->stop) break;
  }
  finish(k + 1);
}

// Tile-edge class of the graphs a launch runs: 0 (T = 128), 1 (64), 2 (32).
template <int T>
struct TileClass {
  static constexpr int v = (T == TILE) ? 0 : (T == 64) ? 1 : 2;
};

// One persistent launch per tile edge present in the batch (all of them in
// one captured CUDA graph): the CTAs take the graphs of class TileClass<T>
// from p.order[cls_off[c] .. cls_off[c + 1]) through queue p.queue[c].
template <int DIM, int W, int T>
__global__ void __launch_bounds__(BGT * W, 1) fd_batch_kernel(const BParams* pp) {
  extern __shared__ __align__(256) unsigned char smem[];
  using SL = BSmem<DIM>;
  constexpr int CLS = TileClass<T>::v;
  {
    static_assert(sizeof(BParams) % 8 == 0, "BParams copy granularity");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(pp);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(smem + SL::OFF_P);
    for (int k = threadIdx.x; k < (int)(sizeof(BParams) / 8); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const BParams& p = *reinterpret_cast<const BParams*>(smem + SL::OFF_P);
  BState* st = reinterpret_cast<BState*>(smem + SL::OFF_ST);
  {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + SL::OFF_MBAR);
    if (threadIdx.x == 0) {
      for (int k = 0; k < BMAX_G * BMAX_NBUF; ++k) mbar_init(&mbar[k], 1);
      fence_mbar_init();
      st->parity = 0u;
    }
    uint4* dst = reinterpret_cast<uint4*>(smem + SL::OFF_LUT);
    const uint4* srcl = reinterpret_cast<const uint4*>(p.lut);
    for (int k = threadIdx.x; k < p.lut_rows * (LUT_ROW / 16); k += blockDim.x) dst[k] = srcl[k];
  }
  __syncthreads();
  __shared__ int s_next;
  const int q0 = p.cls_off[CLS], q1 = p.cls_off[CLS + 1];
  while (true) {
    if (threadIdx.x == 0) s_next = q0 + atomicAdd(p.queue + CLS, 1);
    __syncthreads();
    const int qi = s_next;
    __syncthreads();
    if (qi >= q1) break;
    run_graph<DIM, W, T>(p.order[qi]);
    __syncthreads();
    if (st->abort) {
      if (threadIdx.x == 0) {
        atomicCAS(p.err, 0, (int)E_TIMEOUT);
        p.status[st->graph] = E_TIMEOUT;
      }
      break;
    }
  }
}

}  // namespace fdl
