// fd_apsp.cu -- ideal distances d_ij on the GPU and the row sums of W.
//
// The paper's d_ij is the "predefined ideal distance" of Eq. (1), the
// graph-theoretic shortest-path length as in Gansner et al. (Sec. 2); edges
// of weighted graphs carry lengths (Sec. 5.4).  The CSR edge list is read
// here and nowhere else.
//
// Unit edges: bit-parallel multi-source BFS.  One CTA runs the BFS of 64
// consecutive sources at once; a 64-bit word per vertex holds "reached from
// source b" bits.  Each level pulls the frontier words of a vertex's
// neighbours (one pass over the CSR segment of the vertex), so one pass over
// the edge list advances 64 searches.  Each unordered pair is written once,
// by the source that owns it in the tile layout (fd_internal.cuh).
//
// Weighted edges: one CTA per source runs label-correcting relaxation sweeps
// (dist[v] = min(dist[v], dist[u] + len(u,v))) until no label changes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_internal.cuh"
#include "fd_sssp.cuh"

namespace fdl {

template <int CODE>
__device__ __forceinline__ void put_code(void* D, int tile, int off, float value, int* overflow) {
  if constexpr (CODE == CODE_U8) {
    unsigned char* p = reinterpret_cast<unsigned char*>(D) + (size_t)tile * TILE * TILE + off;
    if (value > 255.f) {
      *p = 255;
      if (overflow) atomicExch(overflow, 1);
    } else {
      *p = (unsigned char)value;
    }
  } else {
    float* p = reinterpret_cast<float*>(D) + (size_t)tile * TILE * TILE + off;
    *p = (value > 0.f) ? __frcp_rn(value) : 0.f;  // float tiles hold 1/d
  }
}

// d of a stored pair (0: no pair or not reached), decoded in FP64.
template <int CODE>
__device__ __forceinline__ double get_code(const void* D, int tile, int off) {
  if constexpr (CODE == CODE_U8) {
    return (double)(reinterpret_cast<const unsigned char*>(D)[(size_t)tile * TILE * TILE + off]);
  } else {
    const float c = reinterpret_cast<const float*>(D)[(size_t)tile * TILE * TILE + off];
    return (c > 0.f) ? 1.0 / (double)c : 0.0;
  }
}

// Bits of a 64-source batch (sources s0 .. s0+63 of block row I) whose pair
// with vertex v is stored by the batch: all bits if v's block is in row I's
// half ring, none if the pair belongs to v's row, and in the diagonal block
// only the sources s < v.
__device__ __forceinline__ unsigned long long owned_bits(int v, int s0, int I, int nb, int LI,
                                                         unsigned long long full, int* k_out) {
  const int J = v / TILE;
  int k = J - I;
  if (k < 0) k += nb;
  *k_out = k;
  if (k == 0) {
    const int dlt = v - s0;
    if (dlt >= 64) return full;
    if (dlt <= 0) return 0ull;
    return ((1ull << dlt) - 1ull) & full;
  }
  return (k < LI) ? full : 0ull;
}

template <int CODE>
__global__ void __launch_bounds__(1024) bfs_batch_kernel(int n, int nb, const int* __restrict__ row_ptr,
                                                         const int* __restrict__ col_idx,
                                                         const int* __restrict__ tile_base,
                                                         const int* __restrict__ strip_len, void* D,
                                                         unsigned long long* scratch, size_t stride,
                                                         int nbatches, int* maxlevel, int* overflow,
                                                         int* sweeps) {
  unsigned long long* vis = scratch + (size_t)blockIdx.x * stride;
  for (int batch = blockIdx.x; batch < nbatches; batch += gridDim.x) {
    unsigned long long* fr = vis + n;
    unsigned long long* nx = fr + n;
    const int s0 = batch * 64;
    const int nsrc = min(64, n - s0);
    const unsigned long long full = (nsrc == 64) ? ~0ull : ((1ull << nsrc) - 1ull);
    const int I = s0 / TILE, il0 = s0 % TILE;
    const int LI = strip_len[I], tb = tile_base[I];
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const unsigned long long b = (v >= s0 && v < s0 + nsrc) ? (1ull << (v - s0)) : 0ull;
      vis[v] = b;
      fr[v] = b;
    }
    __syncthreads();
    int level = 0;
    while (true) {
      ++level;
      int any = 0;
      for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const unsigned long long vs = vis[v];
        unsigned long long nw = 0ull;
        if (vs != full) {
          unsigned long long acc = 0ull;
          const int e1 = row_ptr[v + 1];
          for (int e = row_ptr[v]; e < e1; ++e) acc |= fr[col_idx[e]];
          nw = acc & ~vs & full;
          if (nw) {
            vis[v] = vs | nw;
            any = 1;
            int k;
            unsigned long long m = nw & owned_bits(v, s0, I, nb, LI, full, &k);
            const int jl = v % TILE;
            while (m) {
              const int b = __ffsll((long long)m) - 1;
              m &= m - 1ull;
              put_code<CODE>(D, tb + k, jl * TILE + il0 + b, (float)level, overflow);
            }
          }
        }
        nx[v] = nw;
      }
      any = __syncthreads_or(any);
      if (!any) break;
      unsigned long long* t = fr;
      fr = nx;
      nx = t;
    }
    if (threadIdx.x == 0) {
      atomicMax(maxlevel, level - 1);
      atomicAdd(sweeps, level);  // passes over the edge list, the last (empty) one included
    }
    __syncthreads();
  }
}

// Weighted shortest paths: one source per CTA iteration (frontier search of
// fd_sssp.cuh in the CTA's scratch: 4 n ints), each pair written once into
// the tile that owns it.  *err is set if a search ran out of rounds.
__global__ void __launch_bounds__(1024) sssp_relax_kernel(int n, int nb, const int* __restrict__ row_ptr,
                                                          const int* __restrict__ col_idx,
                                                          const float* __restrict__ len,
                                                          const int* __restrict__ tile_base,
                                                          const int* __restrict__ strip_len, float* D,
                                                          int* scratch, int* maxbits, int* err) {
  __shared__ int s_cnt[2];
  int* dist = scratch + (size_t)blockIdx.x * 4 * n;
  int* mark = dist + n;
  int* fa = mark + n;
  int* fb = fa + n;
  for (int src = blockIdx.x; src < n; src += gridDim.x) {
    if (!sssp_frontier(n, src, row_ptr, col_idx, len, dist, mark, fa, fb, s_cnt) && threadIdx.x == 0)
      atomicExch(err, 1);
    const int I = src / TILE, il = src % TILE;
    const int LI = strip_len[I], tb = tile_base[I];
    int localmax = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const float dv = __int_as_float(__ldcg(dist + v));
      if (v == src || !(dv < INFINITY)) continue;
      const int J = v / TILE;
      int k = J - I;
      if (k < 0) k += nb;
      const bool own = (k == 0) ? (v > src) : (k < LI);
      if (own) D[(size_t)(tb + k) * TILE * TILE + (v % TILE) * TILE + il] = __frcp_rn(dv);  // 1/d
      localmax = max(localmax, __float_as_int(dv));
    }
    atomicMax(maxbits, localmax);
    __syncthreads();
  }
}

// Pairs still holding code 0 after the searches were not reached.  Count
// them and, under policy 1, give them the fill distance.
template <int CODE>
__global__ void fill_unreached_kernel(int n, int nb, int ntiles, const int2* __restrict__ tile_ik, void* D,
                                      float fill, int write, unsigned long long* count) {
  unsigned long long local = 0;
  const size_t total = (size_t)ntiles * TILE * TILE;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int tile = (int)(idx / (TILE * TILE));
    const int off = (int)(idx % (TILE * TILE));
    const int jl = off / TILE, il = off % TILE;
    const int2 ik = tile_ik[tile];
    const int J = (ik.x + ik.y) % nb;
    const int i = ik.x * TILE + il, j = J * TILE + jl;
    const bool real = (i < n) && (j < n) && (ik.y > 0 || il < jl);
    if (real && get_code<CODE>(D, tile, off) == 0.0) {
      ++local;
      if (write) put_code<CODE>(D, tile, off, fill, nullptr);
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// s_i = sum_{j != i} w_ij (diagonal of L^W, Prop. 2.1), FP64 accumulation.
template <int CODE>
__global__ void __launch_bounds__(TILE) rowsum_kernel(int n, int nb, const int* __restrict__ tile_base,
                                                      const int* __restrict__ strip_len, const void* D,
                                                      float* s, float* inv_s) {
  const int R = blockIdx.x, t = threadIdx.x;
  __shared__ double wl[LUT_N];
  if constexpr (CODE == CODE_U8) {
    for (int c = t; c < LUT_N; c += TILE) wl[c] = (c == 0) ? 0.0 : 1.0 / ((double)c * (double)c);
    __syncthreads();
  }
  auto wgt = [&](int tile, int off) -> double {
    if constexpr (CODE == CODE_U8) {
      return wl[reinterpret_cast<const unsigned char*>(D)[(size_t)tile * TILE * TILE + off]];
    } else {
      const double c = reinterpret_cast<const float*>(D)[(size_t)tile * TILE * TILE + off];  // 1/d
      return c * c;  // the weight the pair loop forms, (1/d)^2
    }
  };
  double acc = 0.0;
  // row R as the i side: its own strip, including the diagonal tile (pairs t < jl)
  for (int k = 0; k < strip_len[R]; ++k) {
    const int tile = tile_base[R] + k;
    for (int jl = 0; jl < TILE; ++jl) acc += wgt(tile, jl * TILE + t);
  }
  // row R as the j side: the diagonal tile (pairs il < t) and other strips' tiles
  for (int I = 0; I < nb; ++I) {
    int k = R - I;
    if (k < 0) k += nb;
    if (k >= strip_len[I]) continue;
    const int tile = tile_base[I] + k;
    for (int il = 0; il < TILE; ++il) acc += wgt(tile, t * TILE + il);
  }
  const int i = R * TILE + t;
  s[i] = (float)acc;
  inv_s[i] = (acc > 0.0) ? (float)(1.0 / acc) : 0.f;
}

template <int CODE>
__global__ void distance_rows_kernel(int n, int nb, const int* __restrict__ tile_base,
                                     const int* __restrict__ strip_len, const void* D, int row0, int nrows,
                                     int hop_counts, double* out) {
  const size_t total = (size_t)nrows * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = row0 + (int)(idx / n), j = (int)(idx % n);
    double v = 0.0;
    if (i != j) {
      const int I = i / TILE, J = j / TILE, il = i % TILE, jl = j % TILE;
      if (I == J) {
        const int a = min(il, jl), b = max(il, jl);
        v = get_code<CODE>(D, tile_base[I], b * TILE + a);
      } else {
        int k = J - I;
        if (k < 0) k += nb;
        if (k < strip_len[I]) {
          v = get_code<CODE>(D, tile_base[I] + k, jl * TILE + il);
        } else {
          int k2 = I - J;
          if (k2 < 0) k2 += nb;
          v = get_code<CODE>(D, tile_base[J] + k2, il * TILE + jl);
        }
      }
    }
    // float tiles of a unit-edge graph hold 1/k for a hop count k < 2^24:
    // rounding the decoded value gives k back exactly
    out[idx] = hop_counts ? rint(v) : v;
  }
}

// ------------------------------------------------------------ batched form
//
// Many independent graphs of at most BMAX_N vertices, concatenated: graph g
// owns vertices v0 .. v0 + n - 1 of the shared CSR (every edge stays inside
// its graph) and the tiles t0 .. t0 + hr_tiles(nb) - 1 of the uint8 distance
// pool.  One CTA runs the 64 searches of one work item (graph, first source)
// with the "reached" words in shared memory.

__global__ void __launch_bounds__(512) bfs_multi_kernel(const BGraph* __restrict__ graphs,
                                                        const int2* __restrict__ items, int nitems,
                                                        const int* __restrict__ row_ptr,
                                                        const int* __restrict__ col_idx, unsigned char* D,
                                                        int* maxlevel, int* overflow) {
  extern __shared__ unsigned long long bw[];  // vis[n], fr[n], nx[n]
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const BGraph gr = graphs[item.x];
    const int n = gr.n, nb = gr.nb, v0 = gr.v0, s0 = item.y;
    unsigned long long* vis = bw;
    unsigned long long* fr = bw + n;
    unsigned long long* nx = fr + n;
    const int nsrc = min(64, n - s0);
    const unsigned long long full = (nsrc == 64) ? ~0ull : ((1ull << nsrc) - 1ull);
    const int I = s0 / TILE, il0 = s0 % TILE;
    const int LI = hr_len(nb, I), tb = hr_base(nb, I);
    unsigned char* Dg = D + (size_t)gr.t0 * TILE * TILE;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const unsigned long long b = (v >= s0 && v < s0 + nsrc) ? (1ull << (v - s0)) : 0ull;
      vis[v] = b;
      fr[v] = b;
    }
    __syncthreads();
    int level = 0;
    while (true) {
      ++level;
      int any = 0;
      for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const unsigned long long vs = vis[v];
        unsigned long long nw = 0ull;
        if (vs != full) {
          unsigned long long acc = 0ull;
          const int e1 = row_ptr[v0 + v + 1];
          for (int e = row_ptr[v0 + v]; e < e1; ++e) acc |= fr[col_idx[e] - v0];
          nw = acc & ~vs & full;
          if (nw) {
            vis[v] = vs | nw;
            any = 1;
            int k;
            unsigned long long m = nw & owned_bits(v, s0, I, nb, LI, full, &k);
            const int jl = v % TILE;
            while (m) {
              const int b = __ffsll((long long)m) - 1;
              m &= m - 1ull;
              put_code<CODE_U8>(Dg, tb + k, jl * TILE + il0 + b, (float)level, overflow);
            }
          }
        }
        nx[v] = nw;
      }
      any = __syncthreads_or(any);
      if (!any) break;
      unsigned long long* t = fr;
      fr = nx;
      nx = t;
    }
    if (threadIdx.x == 0) atomicMax(maxlevel + item.x, level - 1);
    __syncthreads();
  }
}

// Unreached pairs of every graph: counted per graph and, under policy 1,
// given the graph's fill distance (largest finite d) + 1.  One CTA per tile.
__global__ void __launch_bounds__(256) fill_multi_kernel(const BGraph* __restrict__ graphs,
                                                         const int* __restrict__ tile_graph,
                                                         const int2* __restrict__ tile_ik, long long ntiles,
                                                         unsigned char* D, const int* __restrict__ maxlevel,
                                                         int write, int* unreached, int* overflow) {
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int g = tile_graph[t];
    const int2 ik = tile_ik[t];
    const BGraph gr = graphs[g];
    const int nb = gr.nb, n = gr.n;
    const int J = (ik.x + ik.y) % nb;
    const float fill = (float)(maxlevel[g] + 1);
    unsigned char* Dt = D + (size_t)t * TILE * TILE;
    int local = 0;
    for (int off = threadIdx.x; off < TILE * TILE; off += blockDim.x) {
      const int jl = off / TILE, il = off % TILE;
      const int i = ik.x * TILE + il, j = J * TILE + jl;
      const bool real = (i < n) && (j < n) && (ik.y > 0 || il < jl);
      if (real && Dt[off] == 0) {
        ++local;
        if (write) {
          if (fill > 255.f) {
            Dt[off] = 255;
            atomicExch(overflow, 1);
          } else {
            Dt[off] = (unsigned char)fill;
          }
        }
      }
    }
    if (local) atomicAdd(unreached + g, local);
  }
}

// s_i = sum_{j != i} w_ij of every graph (FP64 accumulation); work item =
// (graph, block row R), thread t = vertex R * TILE + t.
__global__ void __launch_bounds__(TILE) rowsum_multi_kernel(const BGraph* __restrict__ graphs,
                                                            const int2* __restrict__ items, int nitems,
                                                            const unsigned char* D, float* s, float* inv_s) {
  __shared__ double wl[LUT_N];
  for (int c = threadIdx.x; c < LUT_N; c += TILE) wl[c] = (c == 0) ? 0.0 : 1.0 / ((double)c * (double)c);
  __syncthreads();
  const int t = threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const BGraph gr = graphs[item.x];
    const int nb = gr.nb, R = item.y;
    const unsigned char* Dg = D + (size_t)gr.t0 * TILE * TILE;
    double acc = 0.0;
    for (int k = 0; k < hr_len(nb, R); ++k) {
      const size_t tile = (size_t)hr_base(nb, R) + k;
      for (int jl = 0; jl < TILE; ++jl) acc += wl[Dg[tile * TILE * TILE + jl * TILE + t]];
    }
    for (int I = 0; I < nb; ++I) {
      int k = R - I;
      if (k < 0) k += nb;
      if (k >= hr_len(nb, I)) continue;
      const size_t tile = (size_t)hr_base(nb, I) + k;
      for (int il = 0; il < TILE; ++il) acc += wl[Dg[tile * TILE * TILE + t * TILE + il]];
    }
    const size_t i = (size_t)gr.p0 + R * TILE + t;
    s[i] = (float)acc;
    inv_s[i] = (acc > 0.0) ? (float)(1.0 / acc) : 0.f;
  }
}

// The full distance matrix of one graph of a batch (float64 [n][n], d_ii = 0).
// The stored code of pair (i, j), i != j, of one graph's TILE x TILE half ring.
__device__ __forceinline__ unsigned char code_at(const unsigned char* Dg, int nb, int i, int j) {
  const int I = i / TILE, J = j / TILE, il = i % TILE, jl = j % TILE;
  if (I == J) {
    const int a = min(il, jl), b = max(il, jl);
    return Dg[(size_t)hr_base(nb, I) * TILE * TILE + b * TILE + a];
  }
  int k = J - I;
  if (k < 0) k += nb;
  if (k < hr_len(nb, I)) return Dg[((size_t)hr_base(nb, I) + k) * TILE * TILE + jl * TILE + il];
  int k2 = I - J;
  if (k2 < 0) k2 += nb;
  return Dg[((size_t)hr_base(nb, J) + k2) * TILE * TILE + il * TILE + jl];
}

__global__ void distance_graph_kernel(const unsigned char* Dg, int n, int nb, double* out) {
  const size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    out[idx] = (i != j) ? (double)code_at(Dg, nb, i, j) : 0.0;
  }
}

// The T x T half ring (T = gr.T < TILE, nbt blocks, same layout rules as the
// TILE x TILE one: column-major codes, a diagonal tile holds i < j only, 0 for
// no pair) of each listed graph, from its TILE x TILE tiles.  One CTA per
// graph at a time.
__global__ void __launch_bounds__(256) retile_multi_kernel(const BGraph* __restrict__ graphs,
                                                           const int* __restrict__ list, int count,
                                                           const unsigned char* __restrict__ D,
                                                           unsigned char* __restrict__ DT) {
  for (int li = blockIdx.x; li < count; li += gridDim.x) {
    const BGraph gr = graphs[list[li]];
    const int T = gr.T, nbt = gr.nbt, n = gr.n, TB = T * T;
    const unsigned char* Dg = D + (size_t)gr.t0 * TILE * TILE;
    unsigned char* out = DT + gr.dt;
    int I = 0;
    for (int t = 0; t < hr_tiles(nbt); ++t) {
      while (hr_base(nbt, I + 1) <= t) ++I;
      const int k = t - hr_base(nbt, I);
      const int J = (I + k) % nbt;
      for (int e = threadIdx.x; e < TB; e += blockDim.x) {
        const int jl = e / T, il = e % T;
        const int i = I * T + il, j = J * T + jl;
        unsigned char c = 0;
        if (i < n && j < n && i != j && (k != 0 || i < j)) c = code_at(Dg, gr.nb, i, j);
        out[(size_t)t * TB + e] = c;
      }
    }
  }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_bfs(int code, int n, int nb, const int* rp, const int* ci, const int* tile_base,
                       const int* strip_len, void* D, unsigned long long* scratch, size_t stride, int grid,
                       int* maxlevel, int* overflow, int* sweeps, cudaStream_t st) {
  const int nbatches = (n + 63) / 64;
  if (code == CODE_U8)
    bfs_batch_kernel<CODE_U8><<<grid, 1024, 0, st>>>(n, nb, rp, ci, tile_base, strip_len, D, scratch, stride,
                                                     nbatches, maxlevel, overflow, sweeps);
  else
    bfs_batch_kernel<CODE_F32><<<grid, 1024, 0, st>>>(n, nb, rp, ci, tile_base, strip_len, D, scratch, stride,
                                                      nbatches, maxlevel, overflow, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_sssp(int n, int nb, const int* rp, const int* ci, const float* len, const int* tile_base,
                        const int* strip_len, float* D, int* scratch, int grid, int* maxbits, int* err,
                        cudaStream_t st) {
  sssp_relax_kernel<<<grid, 1024, 0, st>>>(n, nb, rp, ci, len, tile_base, strip_len, D, scratch, maxbits, err);
  return cudaGetLastError();
}

cudaError_t launch_fill(int code, int n, int nb, int ntiles, const int2* tile_ik, void* D, float fill, int write,
                        unsigned long long* count, int grid, cudaStream_t st) {
  if (code == CODE_U8)
    fill_unreached_kernel<CODE_U8><<<grid, 256, 0, st>>>(n, nb, ntiles, tile_ik, D, fill, write, count);
  else
    fill_unreached_kernel<CODE_F32><<<grid, 256, 0, st>>>(n, nb, ntiles, tile_ik, D, fill, write, count);
  return cudaGetLastError();
}

cudaError_t launch_rowsum(int code, int n, int nb, const int* tile_base, const int* strip_len, const void* D,
                          float* s, float* inv_s, cudaStream_t st) {
  if (code == CODE_U8)
    rowsum_kernel<CODE_U8><<<nb, TILE, 0, st>>>(n, nb, tile_base, strip_len, D, s, inv_s);
  else
    rowsum_kernel<CODE_F32><<<nb, TILE, 0, st>>>(n, nb, tile_base, strip_len, D, s, inv_s);
  return cudaGetLastError();
}

cudaError_t launch_distance_rows(int code, int n, int nb, const int* tile_base, const int* strip_len,
                                 const void* D, int row0, int nrows, int hop_counts, double* out, cudaStream_t st) {
  const size_t total = (size_t)nrows * n;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  if (code == CODE_U8)
    distance_rows_kernel<CODE_U8><<<grid, 256, 0, st>>>(n, nb, tile_base, strip_len, D, row0, nrows, 0, out);
  else
    distance_rows_kernel<CODE_F32><<<grid, 256, 0, st>>>(n, nb, tile_base, strip_len, D, row0, nrows, hop_counts,
                                                         out);
  return cudaGetLastError();
}

cudaError_t launch_bfs_multi(const BGraph* graphs, const int2* items, int nitems, const int* rp, const int* ci,
                             unsigned char* D, int n_max, int* maxlevel, int* overflow, int grid, cudaStream_t st) {
  const size_t smem = (size_t)3 * n_max * sizeof(unsigned long long);
  cudaError_t e = cudaFuncSetAttribute(bfs_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  bfs_multi_kernel<<<grid, 512, smem, st>>>(graphs, items, nitems, rp, ci, D, maxlevel, overflow);
  return cudaGetLastError();
}

cudaError_t launch_fill_multi(const BGraph* graphs, const int* tile_graph, const int2* tile_ik, long long ntiles,
                              unsigned char* D, const int* maxlevel, int write, int* unreached, int* overflow, int grid,
                              cudaStream_t st) {
  fill_multi_kernel<<<grid, 256, 0, st>>>(graphs, tile_graph, tile_ik, ntiles, D, maxlevel, write, unreached,
                                          overflow);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_multi(const BGraph* graphs, const int2* items, int nitems, const unsigned char* D, float* s,
                                float* inv_s, int grid, cudaStream_t st) {
  rowsum_multi_kernel<<<grid, TILE, 0, st>>>(graphs, items, nitems, D, s, inv_s);
  return cudaGetLastError();
}

cudaError_t launch_distance_graph(const unsigned char* Dg, int n, int nb, double* out, cudaStream_t st) {
  const size_t total = (size_t)n * n;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  distance_graph_kernel<<<grid, 256, 0, st>>>(Dg, n, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_retile_multi(const BGraph* graphs, const int* list, int count, const unsigned char* D,
                                unsigned char* DT, int grid, cudaStream_t st) {
  retile_multi_kernel<<<grid, 256, 0, st>>>(graphs, list, count, D, DT);
  return cudaGetLastError();
}

}  // namespace fdl
