// fd_grad.cu -- derivative of the stress (Eq. (1)) with respect to the edge
// lengths of a weighted graph.
//
// With w_ij = d_ij^-2 (Sec. 5.1) the pair term is (r_ij / d_ij - 1)^2, so
//     d f / d d_ij = -2 r_ij (r_ij - d_ij) / d_ij^3 =: G_ij,
// and d_ij, the weighted shortest-path length (Sec. 2, Sec. 5.4), moves with
// the length of every edge on the shortest path of (i, j) (ties between
// paths have measure zero for real-valued lengths).  So
//     d f / d l_e = sum over pairs whose shortest path uses e of G_ij.
//
// pair_dgrad_kernel writes G_ij into a float array laid out like the
// distance tiles.  sp_backprop_kernel then takes one source s per CTA
// iteration: label-correcting distances from s in shared memory, the
// shortest-path tree (parent = lowest-index neighbour u with
// dist[u] + l(u, v) == dist[v], an exact FP32 equality at the fixed point),
// a bitonic sort of the vertices by distance, and one sweep from the
// farthest vertex inwards that adds each subtree's sum of G_sv to the
// subtree's parent edge.  Every unordered pair is met from both ends, so the
// per-edge sums are halved when the two directions are combined.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_internal.cuh"
#include "fd_sssp.cuh"

namespace fdl {

__global__ void __launch_bounds__(TILE) pair_dgrad_kernel(int n, int nb, int dim, const int2* __restrict__ tile_ik,
                                                          int ntiles, const float* __restrict__ D,
                                                          const float* __restrict__ X, float* Gt) {
  __shared__ float xi[TILE][3], xj[TILE][3];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 ik = tile_ik[t];
    const int I = ik.x, J = (ik.x + ik.y) % nb;
    const int i = I * TILE + threadIdx.x, j = J * TILE + threadIdx.x;
    for (int d = 0; d < 3; ++d) {
      xi[threadIdx.x][d] = (i < n && d < dim) ? X[(size_t)i * dim + d] : 0.f;
      xj[threadIdx.x][d] = (j < n && d < dim) ? X[(size_t)j * dim + d] : 0.f;
    }
    __syncthreads();
    const int il = threadIdx.x;
    for (int jl = 0; jl < TILE; ++jl) {
      const size_t off = (size_t)t * TILE * TILE + (size_t)jl * TILE + il;
      const float c = D[off];  // 1/d (float tiles)
      float g = 0.f;
      if (c > 0.f) {
        float r2 = 0.f;
        for (int d = 0; d < dim; ++d) {
          const float a = xi[il][d] - xj[jl][d];
          r2 = fmaf(a, a, r2);
        }
        const float r = sqrtf(r2);
        g = -2.f * r * c * c * fmaf(r, c, -1.f);  // -2 r (r - d) / d^3
      }
      Gt[off] = g;
    }
    __syncthreads();
  }
}

// Value of pair (i, j) in an array laid out like the distance tiles.
__device__ __forceinline__ float pair_value(const float* T, int nb, int i, int j) {
  const int I = i / TILE, J = j / TILE, il = i % TILE, jl = j % TILE;
  constexpr size_t TT = (size_t)TILE * TILE;
  if (I == J) {
    const int a = min(il, jl), b = max(il, jl);
    return T[(size_t)hr_base(nb, I) * TT + b * TILE + a];
  }
  int k = J - I;
  if (k < 0) k += nb;
  if (k < hr_len(nb, I)) return T[((size_t)hr_base(nb, I) + k) * TT + jl * TILE + il];
  int k2 = I - J;
  if (k2 < 0) k2 += nb;
  return T[((size_t)hr_base(nb, J) + k2) * TT + il * TILE + jl];
}

__global__ void __launch_bounds__(256) sp_backprop_kernel(int n, int nb, int npow2, const int* __restrict__ rp,
                                                          const int* __restrict__ ci, const float* __restrict__ len,
                                                          const float* __restrict__ Gt, float* gacc) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(sm);  // [npow2]
  float* dist = reinterpret_cast<float*>(key + npow2);                 // [n]
  float* acc = dist + n;                                               // [n]
  int* par_e = reinterpret_cast<int*>(acc + n);                        // [n]
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    for (int v = tid; v < n; v += bd) dist[v] = (v == s) ? 0.f : INFINITY;
    __syncthreads();
    for (int sweep = 0; sweep < n; ++sweep) {
      int changed = 0;
      for (int v = tid; v < n; v += bd) {
        float best = dist[v];
        for (int e = rp[v]; e < rp[v + 1]; ++e) best = fminf(best, ((volatile float*)dist)[ci[e]] + len[e]);
        if (best < dist[v]) {
          dist[v] = best;
          changed = 1;
        }
      }
      if (!__syncthreads_or(changed)) break;
    }
    // shortest-path tree: the lowest-index tight neighbour is the parent
    for (int v = tid; v < n; v += bd) {
      int be = -1, bu = 0x7fffffff;
      if (v != s && dist[v] < INFINITY) {
        for (int e = rp[v]; e < rp[v + 1]; ++e) {
          const int u = ci[e];
          if (u != v && dist[u] + len[e] == dist[v] && u < bu) {
            bu = u;
            be = e;
          }
        }
      }
      par_e[v] = be;
      acc[v] = (v != s) ? pair_value(Gt, nb, s, v) : 0.f;
    }
    for (int v = tid; v < npow2; v += bd)
      key[v] = (v < n && dist[v] < INFINITY) ? (((unsigned long long)__float_as_uint(dist[v]) << 32) | (unsigned)v)
                                              : ~0ull;
    __syncthreads();
    // bitonic sort, ascending distance (non-negative floats order as their bit patterns)
    for (int k = 2; k <= npow2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < npow2; i += bd) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = key[i], b = key[ixj];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              key[i] = b;
              key[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    // farthest first: each subtree's sum reaches its parent edge
    if (tid == 0) {
      for (int k = npow2 - 1; k >= 0; --k) {
        const unsigned long long kk = key[k];
        if (kk == ~0ull) continue;
        const int v = (int)(kk & 0xffffffffull);
        const int e = par_e[v];
        if (v == s || e < 0) continue;
        const float a = acc[v];
        acc[ci[e]] += a;
        atomicAdd(gacc + e, a);
      }
    }
    __syncthreads();
  }
}

// The same back-propagation for graphs whose per-source state does not fit
// shared memory: one source per CTA iteration, 7 n ints of CTA-private
// global scratch.  Distances come from the frontier search (fd_sssp.cuh: the
// same FP32 fixed point as the search that stored them), the parent of v is
// the lowest-index u with dist[u] + l(u, v) == dist[v], and the subtree sums
// move from the leaves to the source in rounds: a vertex joins the next round
// once all of its children have added their sums to it (a count of pending
// children per vertex), so no sort by distance is needed.  Work per source:
// O(n + m), in about as many rounds as the tree is deep.  Scratch accesses
// are L2 (.cg) loads and stores or atomics (atomics never refresh L1).
__global__ void __launch_bounds__(1024) sp_backprop_global_kernel(int n, int nb, const int* __restrict__ rp,
                                                                  const int* __restrict__ ci,
                                                                  const float* __restrict__ len,
                                                                  const float* __restrict__ Gt, float* gacc,
                                                                  int* scratch, int* err) {
  __shared__ int s_cnt[2];
  int* base = scratch + (size_t)blockIdx.x * 7 * n;
  int* dist = base;
  int* mark = base + n;
  int* fa = base + 2 * (size_t)n;
  int* fb = base + 3 * (size_t)n;
  int* par_e = base + 4 * (size_t)n;
  int* pend = base + 5 * (size_t)n;
  float* acc = reinterpret_cast<float*>(base + 6 * (size_t)n);
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    if (!sssp_frontier(n, s, rp, ci, len, dist, mark, fa, fb, s_cnt) && tid == 0) atomicExch(err, 1);
    // shortest-path tree: the lowest-index tight neighbour is the parent
    for (int v = tid; v < n; v += bd) {
      const float dv = __int_as_float(__ldcg(dist + v));
      int be = -1, bu = 0x7fffffff;
      if (v != s && dv < INFINITY) {
        for (int e = rp[v]; e < rp[v + 1]; ++e) {
          const int u = ci[e];
          if (u != v && __int_as_float(__ldcg(dist + u)) + len[e] == dv && u < bu) {
            bu = u;
            be = e;
          }
        }
      }
      __stcg(par_e + v, be);
      __stcg(pend + v, 0);
      __stcg(acc + v, (v != s) ? pair_value(Gt, nb, s, v) : 0.f);
    }
    __syncthreads();
    for (int v = tid; v < n; v += bd) {
      const int e = __ldcg(par_e + v);
      if (e >= 0) atomicAdd(pend + ci[e], 1);
    }
    if (tid == 0) s_cnt[0] = 0;
    __syncthreads();
    // the leaves start
    for (int v = tid; v < n; v += bd)
      if (__ldcg(par_e + v) >= 0 && atomicAdd(pend + v, 0) == 0) __stcg(fa + atomicAdd(s_cnt, 1), v);
    __syncthreads();
    int na = s_cnt[0];
    int* qa = fa;
    int* qb = fb;
    while (na > 0) {  // every vertex joins one round at most: at most n rounds
      if (tid == 0) s_cnt[1] = 0;
      __syncthreads();
      for (int k = tid; k < na; k += bd) {
        const int v = __ldcg(qa + k);
        const int e = __ldcg(par_e + v);
        const int u = ci[e];
        const float a = __ldcg(acc + v);  // final: every child of v added its sum in an earlier round
        atomicAdd(gacc + e, a);
        atomicAdd(acc + u, a);
        if (u != s && atomicSub(pend + u, 1) == 1) __stcg(qb + atomicAdd(s_cnt + 1, 1), u);
      }
      __syncthreads();
      na = s_cnt[1];
      int* t = qa;
      qa = qb;
      qb = t;
      __syncthreads();  // every thread has read the count before it is reset
    }
  }
}

// The undirected edge's derivative from its two CSR entries (each pair was
// met from both ends, hence the half).
__global__ void combine_directions_kernel(int nnz, const int* __restrict__ rev, const float* __restrict__ gacc,
                                          float* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
    out[e] = 0.5f * (gacc[e] + gacc[rev[e]]);
}

// --------------------------------------------------------------------------
// Adjoint of one iteration of Algorithm 2 (lines 4-8), for unrolled
// differentiation.  Forward: b = L^X X (Prop. 2.1), Y solves L^W Y = b,
// Z = Y - 1 y_0^T (pinning), X' = (1 + omega) Z - omega X if line 6 accepted
// the extrapolation (Eq. (10)), else X' = Z.  The acceptance decision is held
// fixed.  Backward, from Xb' = dL/dX':
//   Zb = (1 + omega) Xb' or Xb';  Xb = -omega Xb' or 0
//   Yb = Zb - e_0 (1^T Zb)                   (adjoint of the pinning)
//   L^W lam = Yb                             (KM_SOLVE of the layout kernel)
//   Xb += J_b(X)^T lam,  per pair: (1/(d r)) (dlam - u (u . dlam)) to i, minus that to j
//   db_ij += -(dlam . u) / d^2 + 2 (dlam . dY) / d^3   (through b and through L^W)
// with u = (x_i - x_j)/r, dlam = lam_i - lam_j, dY = Y_i - Y_j.
// --------------------------------------------------------------------------

// One CTA: Z (recovered from X' and X), the right-hand side Yb of the adjoint
// solve, and the part of Xb that does not pass through the solve.
__global__ void __launch_bounds__(1024) adjoint_prep_kernel(int n, int dim, const float* __restrict__ Xk,
                                                            const float* __restrict__ Xk1, const float* __restrict__ Xb1,
                                                            int accepted, float omega,
                                                            const float* __restrict__ oms, float* Y, float* Yb,
                                                            float* Xb) {
  __shared__ double part[32][3];
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    // omega_i = omega m_i with per-vertex factors (Sec. 6), as in the forward step
    const float om = oms ? omega * oms[i] : omega;
    const float zs = accepted ? 1.f + om : 1.f;
    for (int d = 0; d < dim; ++d) {
      const size_t k = (size_t)i * dim + d;
      const float xb1 = Xb1[k];
      Y[k] = accepted ? (Xk1[k] + om * Xk[k]) / (1.f + om) : Xk1[k];
      const float zb = zs * xb1;
      Yb[k] = zb;
      Xb[k] = accepted ? -om * xb1 : 0.f;
      s[d] += (double)zb;
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) s[d] += __shfl_down_sync(0xffffffffu, s[d], o);
  if ((threadIdx.x & 31) == 0)
    for (int d = 0; d < 3; ++d) part[threadIdx.x >> 5][d] = s[d];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int d = 0; d < dim; ++d) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][d];
      Yb[d] = (float)((double)Yb[d] - t);  // vertex 0 is pinned
    }
  }
}

// One CTA per tile: the vector-Jacobian product of b = L^X X with lam, and
// the pair sensitivities, added to Xb (atomics) and to the float tile array Db.
template <int CODE>
__global__ void __launch_bounds__(TILE) pair_adjoint_kernel(int n, int nb, int dim, const int2* __restrict__ tile_ik,
                                                            int ntiles, const void* __restrict__ D,
                                                            const float* __restrict__ X, const float* __restrict__ lam,
                                                            const float* __restrict__ Y, float* Xb, float* Db) {
  __shared__ float xi[TILE][3], xj[TILE][3], li[TILE][3], lj[TILE][3], yi[TILE][3], yj[TILE][3];
  __shared__ float colacc[TILE][3];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 ik = tile_ik[t];
    const int I = ik.x, J = (ik.x + ik.y) % nb;
    const int i = I * TILE + threadIdx.x, j = J * TILE + threadIdx.x;
    for (int d = 0; d < 3; ++d) {
      const bool ri = (i < n && d < dim), rj = (j < n && d < dim);
      xi[threadIdx.x][d] = ri ? X[(size_t)i * dim + d] : 0.f;
      xj[threadIdx.x][d] = rj ? X[(size_t)j * dim + d] : 0.f;
      li[threadIdx.x][d] = ri ? lam[(size_t)i * dim + d] : 0.f;
      lj[threadIdx.x][d] = rj ? lam[(size_t)j * dim + d] : 0.f;
      yi[threadIdx.x][d] = ri ? Y[(size_t)i * dim + d] : 0.f;
      yj[threadIdx.x][d] = rj ? Y[(size_t)j * dim + d] : 0.f;
      colacc[threadIdx.x][d] = 0.f;
    }
    __syncthreads();
    const int il = threadIdx.x;
    float rowacc[3] = {0.f, 0.f, 0.f};
    for (int jj = 0; jj < TILE; ++jj) {
      const int jl = (il + jj) & (TILE - 1);  // rotate the columns so that the shared-memory atomics spread
      const size_t off = (size_t)t * TILE * TILE + (size_t)jl * TILE + il;
      float inv_d;  // 1/d: from the hop count, or stored in float tiles
      if constexpr (CODE == CODE_U8) {
        const float dd = (float)reinterpret_cast<const unsigned char*>(D)[off];
        inv_d = (dd > 0.f) ? 1.f / dd : 0.f;
      } else {
        inv_d = reinterpret_cast<const float*>(D)[off];
      }
      if (!(inv_d > 0.f)) continue;
      float dx[3], dl[3], r2 = 0.f, ul = 0.f, ly = 0.f;
      for (int d = 0; d < dim; ++d) {
        dx[d] = xi[il][d] - xj[jl][d];
        dl[d] = li[il][d] - lj[jl][d];
        r2 = fmaf(dx[d], dx[d], r2);
        ly = fmaf(dl[d], yi[il][d] - yj[jl][d], ly);
      }
      float g = 2.f * ly * inv_d * inv_d * inv_d;  // through w = d^-2 in L^W
      if (r2 > 0.f) {
        const float r = sqrtf(r2), inv_r = 1.f / r;
        for (int d = 0; d < dim; ++d) ul = fmaf(dx[d] * inv_r, dl[d], ul);
        g -= ul * inv_d * inv_d;  // through the coefficient 1/d of b
        const float c = inv_d * inv_r;
        for (int d = 0; d < dim; ++d) {
          const float v = c * (dl[d] - dx[d] * inv_r * ul);
          rowacc[d] += v;
          atomicAdd(&colacc[jl][d], -v);
        }
      }
      if (Db) Db[off] += g;
    }
    __syncthreads();
    if (i < n)
      for (int d = 0; d < dim; ++d) atomicAdd(Xb + (size_t)i * dim + d, rowacc[d]);
    if (j < n)
      for (int d = 0; d < dim; ++d) atomicAdd(Xb + (size_t)j * dim + d, colacc[threadIdx.x][d]);
    __syncthreads();
  }
}

cudaError_t launch_adjoint_prep(int n, int dim, const float* Xk, const float* Xk1, const float* Xb1, int accepted,
                                float omega, const float* oms, float* Y, float* Yb, float* Xb, cudaStream_t st) {
  adjoint_prep_kernel<<<1, 1024, 0, st>>>(n, dim, Xk, Xk1, Xb1, accepted, omega, oms, Y, Yb, Xb);
  return cudaGetLastError();
}

cudaError_t launch_pair_adjoint(int code, int n, int nb, int dim, const int2* tile_ik, int ntiles, const void* D,
                                const float* X, const float* lam, const float* Y, float* Xb, float* Db, int sm_count,
                                cudaStream_t st) {
  const int grid = ntiles < 8 * sm_count ? ntiles : 8 * sm_count;
  if (code == CODE_U8)
    pair_adjoint_kernel<CODE_U8><<<grid > 0 ? grid : 1, TILE, 0, st>>>(n, nb, dim, tile_ik, ntiles, D, X, lam, Y, Xb, Db);
  else
    pair_adjoint_kernel<CODE_F32><<<grid > 0 ? grid : 1, TILE, 0, st>>>(n, nb, dim, tile_ik, ntiles, D, X, lam, Y, Xb, Db);
  return cudaGetLastError();
}

// Shortest-path back-propagation of an array of pair sensitivities (tile
// layout) to the edges: in shared memory per source up to SP_SMEM_MAX_N
// vertices (unless global_path), else with global scratch (scratch:
// [min(n, 2 SMs)][7 n] ints; err: one int, set if a search ran out of rounds).
constexpr int SP_SMEM_MAX_N = 4096;

size_t sp_backprop_scratch_ints(int n, int sm_count) {
  const int grid = n < 2 * sm_count ? n : 2 * sm_count;
  return (size_t)grid * 7 * (size_t)n;
}

static cudaError_t sp_backprop_run(int n, int nb, const float* Gt, const int* rp, const int* ci, const float* len,
                                   const int* rev, int nnz, float* gacc, float* out, int sm_count, int global_path,
                                   int* scratch, int* err, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(gacc, 0, (size_t)nnz * sizeof(float), st);
  if (e != cudaSuccess) return e;
  const int sgrid = n < 2 * sm_count ? n : 2 * sm_count;
  if (!global_path && n <= SP_SMEM_MAX_N) {
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    const size_t smem = (size_t)npow2 * 8 + (size_t)n * 12;
    e = cudaFuncSetAttribute(sp_backprop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sp_backprop_kernel<<<sgrid, 256, smem, st>>>(n, nb, npow2, rp, ci, len, Gt, gacc);
  } else {
    if (!scratch || !err) return cudaErrorInvalidValue;
    sp_backprop_global_kernel<<<sgrid, 1024, 0, st>>>(n, nb, rp, ci, len, Gt, gacc, scratch, err);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int cgrid = (nnz + 255) / 256;
  if (nnz > 0) combine_directions_kernel<<<cgrid < 4096 ? cgrid : 4096, 256, 0, st>>>(nnz, rev, gacc, out);
  return cudaGetLastError();
}

cudaError_t launch_sp_backprop(int n, int nb, const float* Gt, const int* rp, const int* ci, const float* len,
                               const int* rev, int nnz, float* gacc, float* out, int sm_count, int global_path,
                               int* scratch, int* err, cudaStream_t st) {
  return sp_backprop_run(n, nb, Gt, rp, ci, len, rev, nnz, gacc, out, sm_count, global_path, scratch, err, st);
}

cudaError_t launch_length_grad(int n, int nb, int dim, const int2* tile_ik, int ntiles, const float* D,
                               const float* X, float* Gt, const int* rp, const int* ci, const float* len,
                               const int* rev, int nnz, float* gacc, float* out, int sm_count, int global_path,
                               int* scratch, int* err, cudaStream_t st) {
  const int tgrid = ntiles < 8 * sm_count ? ntiles : 8 * sm_count;
  pair_dgrad_kernel<<<tgrid > 0 ? tgrid : 1, TILE, 0, st>>>(n, nb, dim, tile_ik, ntiles, D, X, Gt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sp_backprop_run(n, nb, Gt, rp, ci, len, rev, nnz, gacc, out, sm_count, global_path, scratch, err, st);
}

}  // namespace fdl
