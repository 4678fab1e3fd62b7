// fd_sssp.cuh -- single-source shortest paths over positive edge lengths,
// one CTA per source, for the weighted ideal distances (Sec. 2: d_ij is the
// shortest-path length; weighted edges as for the railway net of Sec. 5.4).
//
// Frontier (push) label correction: a round relaxes the edges out of the
// vertices whose distance improved in the round before, with an integer
// atomicMin on the bit patterns (non-negative floats order like their bits).
// For positive lengths every label-correcting order reaches the same FP32
// fixed point -- each vertex's value is the least left-to-right FP32 sum
// over its paths -- so a recomputed search reproduces a stored one bit for
// bit, which the tight-parent test of the length derivative relies on.
// Membership of the next frontier is stamped with the round number, so a
// vertex improved twice in a round is queued once and one improved while
// being relaxed is queued again, with no flag to clear.
#pragma once

#include "fd_internal.cuh"

namespace fdl {

constexpr int SSSP_INF_BITS = 0x7f800000;  // +inf

// dist, mark, fa, fb: [n] ints of CTA-private global scratch; s_cnt: two
// shared ints.  On return (every thread) dist holds the distances as float
// bits; false if the round limit ran out (then dist is incomplete).  The
// scratch is only touched by atomics and L2 (.cg) loads and stores: atomics
// are performed in L2 and never refresh a line an SM holds in L1.
__device__ __forceinline__ bool sssp_frontier(int n, int s, const int* __restrict__ rp, const int* __restrict__ ci,
                                              const float* __restrict__ len, int* dist, int* mark, int* fa, int* fb,
                                              int* s_cnt) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int v = tid; v < n; v += bd) {
    __stcg(dist + v, (v == s) ? 0 : SSSP_INF_BITS);
    __stcg(mark + v, 0);
  }
  if (tid == 0) {
    __stcg(fa, s);
    s_cnt[0] = 1;
  }
  __syncthreads();
  int na = s_cnt[0];
  int round = 0;
  bool ok = true;
  while (na > 0) {
    ++round;
    if (round > 4 * n + 16) {  // far beyond any real search: give up (uniform over the CTA)
      ok = false;
      break;
    }
    if (tid == 0) s_cnt[1] = 0;
    __syncthreads();
    for (int k = tid; k < na; k += bd) {
      const int u = __ldcg(fa + k);
      const float du = __int_as_float(__ldcg(dist + u));
      const int e1 = rp[u + 1];
      for (int e = rp[u]; e < e1; ++e) {
        const int v = ci[e];
        const int nd = __float_as_int(du + len[e]);
        if (nd < atomicMin(dist + v, nd)) {
          if (atomicExch(mark + v, round) != round) __stcg(fb + atomicAdd(s_cnt + 1, 1), v);
        }
      }
    }
    __syncthreads();
    na = s_cnt[1];
    int* t = fa;
    fa = fb;
    fb = t;
    __syncthreads();  // every thread has read the count before it is reset
  }
  return ok;
}

}  // namespace fdl
