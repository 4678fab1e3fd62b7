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

// Breadth-first searches for large graphs of small diameter.  bfs_batch_kernel
// gives each CTA a 64-source batch of its own, and at n = 200,000 the CTAs'
// per-vertex words (3 x 8 B x n each, 1.5 GB over 304 CTAs) overflow L2, so
// every 8-byte neighbour-word gather costs a 32-byte DRAM sector.  Here all
// CTAs take one batch of 256 sources at a time (a 32-byte word per vertex and
// level) level by level, with a grid barrier (bounded waits) after each
// level, so the words stay in L2.  A level costs a grid barrier, so this pays
// for graphs with few levels per search (chosen on the host).
//
// Words: vis (sources that reached v) and the frontier F_l (sources that
// reached v at level l) of every level l <= lcap, kept to the end of the
// batch; deeper levels alternate between two further slots.  The 1-byte
// codes of levels <= lcap are written at the end of the batch, 16 sources per
// 16-byte store (the byte d_sv of source s is l for the l whose F_l holds s),
// instead of one byte store per pair as each is reached; codes of deeper
// levels (and float codes) are written as reached.
//
// A level ends with its slowest vertex, so vertices of degree above
// WIDE_BIG_DEG are pulled by a warp each, the lanes striding over the edges
// (tasks[] from the host, largest degree first), the others by a thread
// each; a vertex of degree above WIDE_HUB_CHUNK (a hub) is split into tasks
// of WIDE_HUB_CHUNK edges, whose warps OR their partial words into the
// hub's word and the last of which finishes the vertex.  A batch ends after
// the level that reached nothing or the level after which every vertex
// holds every source.
constexpr int WIDE_BIG_DEG = 16;
constexpr int WIDE_HUB_CHUNK = 256;

struct __align__(32) Words4 {
  unsigned long long w[4];
};

__device__ __forceinline__ void or_word(Words4& acc, const Words4* f) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(f);
  const ulonglong2 lo = __ldcg(q), hi = __ldcg(q + 1);
  acc.w[0] |= lo.x;
  acc.w[1] |= lo.y;
  acc.w[2] |= hi.x;
  acc.w[3] |= hi.y;
}

// acc |= fr[col_idx[e]] over e = e0, e0 + st, .. < e1, four gathers in flight
// (a level lasts as long as its slowest vertex's chain of L2 round trips).
__device__ __forceinline__ void gather_or(Words4& acc, const Words4* fr, const int* __restrict__ col_idx, int e0,
                                          int e1, int st) {
  int e = e0;
  for (; e + 3 * st < e1; e += 4 * st) {
    const int u0 = col_idx[e], u1 = col_idx[e + st], u2 = col_idx[e + 2 * st], u3 = col_idx[e + 3 * st];
    or_word(acc, fr + u0);
    or_word(acc, fr + u1);
    or_word(acc, fr + u2);
    or_word(acc, fr + u3);
  }
  for (; e < e1; e += st) or_word(acc, fr + col_idx[e]);
}

// Codes of the sources of word w (sources s0 + 64 w ..) in the bits of nw
// (reached v at this level) whose pair with v the batch's strips store.
template <int CODE>
__device__ __forceinline__ void wide_codes(void* D, int v, int s0, int w, unsigned long long nw, int nb,
                                           const int* __restrict__ tile_base, const int* __restrict__ strip_len,
                                           unsigned long long full, int level, int* overflow) {
  const int sw = s0 + 64 * w, I = sw / TILE, il0 = sw % TILE;
  int k;
  unsigned long long m = nw & owned_bits(v, sw, I, nb, strip_len[I], full, &k);
  if (!m) return;
  const int tb = tile_base[I], jl = v % TILE;
  while (m) {
    const int b = __ffsll((long long)m) - 1;
    m &= m - 1ull;
    put_code<CODE>(D, tb + k, jl * TILE + il0 + b, (float)level, overflow);
  }
}

// Frontier slot of level l: l itself up to lcap, then two alternating slots.
__device__ __forceinline__ int wide_slot(int l, int lcap) { return (l <= lcap) ? l : lcap + 1 + (l & 1); }

// acc |= (the bits of the batch's sources s0 .. s0 + nsrc - 1 among col_idx[e],
// e = e0, e0 + st, .. < e1): the frontier of level 0 without reading it.
__device__ __forceinline__ void source_or(Words4& acc, const int* __restrict__ col_idx, int e0, int e1, int st,
                                          int s0, int nsrc) {
  for (int e = e0; e < e1; e += st) {
    const int d = col_idx[e] - s0;
    if (d >= 0 && d < nsrc) {
      const unsigned long long bit = 1ull << (d & 63);
      const int w = d >> 6;  // register selects, not a local-memory index
      acc.w[0] |= (w == 0) ? bit : 0ull;
      acc.w[1] |= (w == 1) ? bit : 0ull;
      acc.w[2] |= (w == 2) ? bit : 0ull;
      acc.w[3] |= (w == 3) ? bit : 0ull;
    }
  }
}

// Grid barrier b of the level loop, fused with the OR of two per-CTA flags
// (bit 0: a vertex was reached at this level; bit 1: a vertex is still
// unreached by some source).  Slot b mod 3 of bar3 counts arrivals in bits
// 0-20, flag-0 CTAs in bits 21-41, flag-1 CTAs in bits 42-62; CTA 0 clears
// slot b + 1 before it arrives at b (its last readers arrived at b - 1).
// Returns the two ORed flags, or -1 after a wait of timeout_ns (E_TIMEOUT
// recorded) or another CTA's error.
__device__ __forceinline__ int wide_barrier(unsigned long long* bar3, int b, int flags, Ctrl* ctrl,
                                            long long timeout_ns) {
  __shared__ int s_res;
  const int f0 = __syncthreads_or(flags & 1), f1 = __syncthreads_or(flags & 2);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) atomicExch(bar3 + (b + 1) % 3, 0ull);
    __threadfence();
    atomicAdd(bar3 + b % 3, 1ull + (f0 ? (1ull << 21) : 0ull) + (f1 ? (1ull << 42) : 0ull));
    volatile unsigned long long* slot = bar3 + b % 3;
    volatile int* err = &ctrl->err;
    unsigned long long v = *slot;
    int res = 0;
    if ((v & 0x1fffffull) != gridDim.x) {
      const unsigned long long t0 = globaltimer_ns();
      while (true) {
        v = *slot;
        if ((v & 0x1fffffull) == gridDim.x) break;
        if (*err != 0) {
          res = -1;
          break;
        }
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
          atomicCAS(&ctrl->err, 0, (int)E_TIMEOUT);
          atomicExch(&ctrl->timeout_where, b);
          res = -1;
          break;
        }
      }
    }
    __threadfence();
    if (res == 0) res = (((v >> 21) & 0x1fffffull) ? 1 : 0) | (((v >> 42) & 0x1fffffull) ? 2 : 0);
    s_res = res;
  }
  __syncthreads();
  return s_res;
}

// 1-byte codes of vertex v's pairs with the sources of word w (s0 + 64 w ..)
// from the frontiers F_1 .. F_lmax (disjoint bit sets): byte b of a 16-source
// group is l where bit b is in F_l, 0 where no F_l holds it (unreached, filled
// later; or reached below level lmax, written as reached: merge ORs the stored
// bytes in, each byte being nonzero on one side at most).
// spread[x]: byte i is 1 where bit i of x is set.
__device__ __forceinline__ void wide_decode_word(unsigned char* D, int v, int s0, int w, unsigned long long fw,
                                              const Words4* __restrict__ F, int n, int lmax, bool merge, int nb,
                                              const int* __restrict__ tile_base,
                                              const int* __restrict__ strip_len,
                                              const unsigned long long* spread) {
  if (!fw) return;
  const int sw = s0 + 64 * w, I = sw / TILE, il0 = sw % TILE;
  int k;
  const unsigned long long om = owned_bits(v, sw, I, nb, strip_len[I], fw, &k);
  if (!om) return;
  unsigned long long c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) c[q] = 0ull;
  auto level_bytes = [&](unsigned long long x, int l) {
    if (!x) return;
    const unsigned long long lv = (unsigned long long)l;
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] |= spread[(x >> (8 * q)) & 0xff] * lv;
  };
  const unsigned long long* Fw = &F[v].w[w];  // F_l's word w of v: Fw[4 n l]
  int l = 1;
  for (; l + 3 <= lmax; l += 4) {  // four loads in flight
    const unsigned long long x0 = __ldcg(Fw + (size_t)4 * n * l), x1 = __ldcg(Fw + (size_t)4 * n * (l + 1)),
                             x2 = __ldcg(Fw + (size_t)4 * n * (l + 2)), x3 = __ldcg(Fw + (size_t)4 * n * (l + 3));
    level_bytes(x0, l);
    level_bytes(x1, l + 1);
    level_bytes(x2, l + 2);
    level_bytes(x3, l + 3);
  }
  for (; l <= lmax; ++l) level_bytes(__ldcg(Fw + (size_t)4 * n * l), l);
  unsigned char* row = D + (size_t)(tile_base[I] + k) * TILE * TILE + (v % TILE) * TILE + il0;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const unsigned gm = (unsigned)(om >> (16 * g)) & 0xffffu;
    if (gm == 0xffffu) {
      ulonglong2* p = reinterpret_cast<ulonglong2*>(row + 16 * g);
      if (merge) {
        const ulonglong2 o = *p;
        *p = make_ulonglong2(c[2 * g] | o.x, c[2 * g + 1] | o.y);
      } else {
        *p = make_ulonglong2(c[2 * g], c[2 * g + 1]);
      }
    } else if (gm) {  // the diagonal block or the ragged last batch: owned bytes only
      for (int b = 0; b < 16; ++b) {
        const unsigned char cb = (unsigned char)(c[2 * g + (b >> 3)] >> (8 * (b & 7)));
        if (((gm >> b) & 1u) && (cb || !merge)) row[16 * g + b] = cb;
      }
    }
  }
}

__device__ __forceinline__ unsigned long long pick4(const unsigned long long* a, int w) {
  return (w == 0) ? a[0] : (w == 1) ? a[1] : (w == 2) ? a[2] : a[3];  // register selects
}

// Sources s0 + 64 w .. of a batch of nsrc sources, as bits of word w.
__device__ __forceinline__ unsigned long long wide_full(int nsrc, int w) {
  const int c = min(64, max(0, nsrc - 64 * w));
  return (c == 64) ? ~0ull : ((1ull << c) - 1ull);
}

// The batch's own bits of vertex v (its level-0 frontier).
__device__ __forceinline__ Words4 self_bits(int v, int s0, int nsrc) {
  Words4 b;
  const int d = v - s0;
#pragma unroll
  for (int w = 0; w < 4; ++w) b.w[w] = (d >= 64 * w && d < 64 * w + 64 && d < nsrc) ? (1ull << (d & 63)) : 0ull;
  return b;
}

template <int CODE>
__global__ void __launch_bounds__(512, 2) bfs_wide_kernel(int n, int nb, const int* __restrict__ row_ptr,
                                                           const int* __restrict__ col_idx,
                                                           const int* __restrict__ tile_base,
                                                           const int* __restrict__ strip_len, void* D,
                                                           Words4* words, int lcap, const int4* __restrict__ tasks,
                                                           int ntasks, Words4* hubacc, int* hubcnt,
                                                           const int* __restrict__ hubparts, int nhub,
                                                           unsigned long long* bar3, Ctrl* ctrl,
                                                           long long timeout_ns, int* maxlevel, int* overflow,
                                                           int* sweeps) {
  __shared__ unsigned long long spread[256];
  for (int x = threadIdx.x; x < 256; x += blockDim.x) {
    unsigned long long e = 0ull;
    for (int i = 0; i < 8; ++i)
      if ((x >> i) & 1) e |= 1ull << (8 * i);
    spread[x] = e;
  }
  __syncthreads();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, nwarps = gstride >> 5, twarp = (gstride - 1 - gtid) >> 5;
  const int nbatches = (n + 255) / 256;
  Words4* vis = words;
  Words4* F = words + n;  // [lcap + 3][n]; slot 0 unused (level 1 reads col_idx alone)
  int b = 0;
  for (int batch = 0; batch < nbatches; ++batch) {
    const int s0 = batch * 256;
    const int nsrc = min(256, n - s0);
    // full_at(w): the batch's sources in word w, recomputed where used (registers)
#define full_at(w) wide_full(nsrc, (w))
    // Every vertex's words (vis, F_l) are written only by its own agent (the
    // thread or warp below, the same in every batch and level), so a batch
    // starts without a barrier: its level 1 reads no frontier.
    int level = 0, deepest = 0;
    while (true) {
      ++level;
      const Words4* fr = F + (size_t)wide_slot(level - 1, lcap) * n;
      Words4* nx = F + (size_t)wide_slot(level, lcap) * n;
      const bool now = (CODE != CODE_U8) || level > lcap;  // codes written as reached
      int any = 0, open_after = 0;
      // vertices of degree <= WIDE_BIG_DEG: a thread each
      for (int v = gtid; v < n; v += gstride) {
        const int e0 = row_ptr[v], e1 = row_ptr[v + 1];
        if (e1 - e0 > WIDE_BIG_DEG) continue;
        const Words4 vs = (level == 1) ? self_bits(v, s0, nsrc) : vis[v];
        Words4 nw;
        bool open = false;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          nw.w[w] = 0ull;
          open = open || (vs.w[w] != full_at(w));
        }
        Words4 nv = vs;
        if (open) {
          Words4 acc;
#pragma unroll
          for (int w = 0; w < 4; ++w) acc.w[w] = 0ull;
          if (level == 1)
            source_or(acc, col_idx, e0, e1, 1, s0, nsrc);
          else
            gather_or(acc, fr, col_idx, e0, e1, 1);
          bool got = false, still = false;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            nw.w[w] = acc.w[w] & ~vs.w[w] & full_at(w);
            nv.w[w] = vs.w[w] | nw.w[w];
            got = got || (nw.w[w] != 0ull);
            still = still || (nv.w[w] != full_at(w));
          }
          if (still) open_after = 2;
          if (got) {
            any = 1;
            if (now) {
#pragma unroll
              for (int w = 0; w < 4; ++w)
                if (nw.w[w])
                  wide_codes<CODE>(D, v, s0, w, nw.w[w], nb, tile_base, strip_len, full_at(w), level, overflow);
            }
          }
          if (got || level == 1) vis[v] = nv;
        } else if (level == 1) {
          vis[v] = vs;
        }
        nx[v] = nw;
      }
      // vertices of larger degree: a task per warp, (v, first edge, end,
      // hub): hub -1 for a whole vertex, else 2 h + (1 for the hub's first
      // task).  The warp that finishes a vertex (the whole-vertex one, or a
      // hub's last) writes its words; lane l then writes the codes of bits
      // [8 (l % 8), 8 (l % 8) + 8) of word l / 8.  vis[v] of a hub is
      // written by whichever warp finishes it: read past L1.  Tasks go to
      // the warps from the last one down (twarp), so the largest ones land
      // on warps whose threads hold one small vertex, not two.
      for (int i = twarp; i < ntasks; i += nwarps) {
        const int4 tk = tasks[i];
        const int v = tk.x, hub = tk.w;
        Words4 vs;
        if (level == 1) {
          vs = self_bits(v, s0, nsrc);
        } else {
          const ulonglong2* q = reinterpret_cast<const ulonglong2*>(vis + v);
          const ulonglong2 lo = __ldcg(q), hi = __ldcg(q + 1);
          vs.w[0] = lo.x;
          vs.w[1] = lo.y;
          vs.w[2] = hi.x;
          vs.w[3] = hi.y;
        }
        bool open = false;
#pragma unroll
        for (int w = 0; w < 4; ++w) open = open || (vs.w[w] != full_at(w));
        Words4 nw;
#pragma unroll
        for (int w = 0; w < 4; ++w) nw.w[w] = 0ull;
        Words4 nv = vs;
        bool finish = (hub < 0) || (!open && (hub & 1));  // warp-uniform
        if (open) {  // warp-uniform (every task of a hub reads the same vis)
          Words4 acc;
#pragma unroll
          for (int w = 0; w < 4; ++w) acc.w[w] = 0ull;
          if (level == 1)
            source_or(acc, col_idx, tk.y + lane, tk.z, 32, s0, nsrc);
          else
            gather_or(acc, fr, col_idx, tk.y + lane, tk.z, 32);
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)acc.w[w]);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(acc.w[w] >> 32));
            acc.w[w] = ((unsigned long long)hi << 32) | lo;
          }
          if (hub >= 0) {
            const int h = hub >> 1;
            int last = 0;
            if (lane == 0) {
#pragma unroll
              for (int w = 0; w < 4; ++w)
                if (acc.w[w]) atomicOr(&hubacc[h].w[w], acc.w[w]);
              __threadfence();
              last = (atomicAdd(hubcnt + h, 1) == hubparts[h] - 1);
            }
            finish = __shfl_sync(0xffffffffu, last, 0) != 0;
            if (finish) {  // every other task of the hub has added its words
              __threadfence();
              const ulonglong2* q = reinterpret_cast<const ulonglong2*>(hubacc + h);
              const ulonglong2 lo = __ldcg(q), hi = __ldcg(q + 1);
              acc.w[0] = lo.x;
              acc.w[1] = lo.y;
              acc.w[2] = hi.x;
              acc.w[3] = hi.y;
              __syncwarp();
              if (lane == 0) {  // ready for the next level (after the grid barrier)
                hubacc[h] = Words4{{0ull, 0ull, 0ull, 0ull}};
                hubcnt[h] = 0;
              }
            }
          }
          if (finish) {
            bool got = false, still = false;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              nw.w[w] = acc.w[w] & ~vs.w[w] & full_at(w);
              nv.w[w] = vs.w[w] | nw.w[w];
              got = got || (nw.w[w] != 0ull);
              still = still || (nv.w[w] != full_at(w));
            }
            if (still) open_after = 2;
            if (got) {
              any = 1;
              if (now) {
                const int w = lane >> 3;
                const unsigned long long mine = pick4(nw.w, w) & (0xffull << (8 * (lane & 7)));
                if (mine)
                  wide_codes<CODE>(D, v, s0, w, mine, nb, tile_base, strip_len, full_at(w), level, overflow);
              }
            }
          }
        }
        if (finish && lane == 0) {
          if (open || level == 1) vis[v] = nv;
          nx[v] = nw;
        }
      }
      const int res = wide_barrier(bar3, b++, any | open_after, ctrl, timeout_ns);
      if (res < 0) return;
      if (!(res & 1)) {  // nothing reached at this level: the previous one was the last
        deepest = level - 1;
        break;
      }
      if (!(res & 2)) {  // every vertex reached by every source
        deepest = level;
        break;
      }
    }
    if constexpr (CODE == CODE_U8) {
      // codes of levels 1 .. min(deepest, lcap), each vertex by its own agent
      const int lmax = min(deepest, lcap);
      const bool merge = deepest > lcap;
      unsigned char* Du = reinterpret_cast<unsigned char*>(D);
      for (int v = gtid; v < n; v += gstride) {
        if (row_ptr[v + 1] - row_ptr[v] > WIDE_BIG_DEG) continue;
        for (int w = 0; w < 4; ++w)
          wide_decode_word(Du, v, s0, w, full_at(w), F, n, lmax, merge, nb, tile_base, strip_len, spread);
      }
      for (int i = twarp; i < ntasks; i += nwarps) {
        const int4 tk = tasks[i];
        if (lane < 4 && (tk.w < 0 || (tk.w & 1)))  // a hub by the warp of its first task
          wide_decode_word(Du, tk.x, s0, lane, full_at(lane), F, n, lmax, merge, nb, tile_base, strip_len,
                           spread);
      }
      // a hub's words of the next batch's level 1 are written by whichever
      // warp finishes it, possibly another than the one that just read them
      if (nhub > 0 && wide_barrier(bar3, b++, 0, ctrl, timeout_ns) < 0) return;
    }
#undef full_at
    if (gtid == 0) {
      atomicMax(maxlevel, deepest);
      atomicAdd(sweeps, level);  // passes over the edge list
    }
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

// Cooperative launch of bfs_wide_kernel (every CTA resident): words
// [lcap + 4][n] Words4 (vis, then the frontier slots); lcap: frontiers kept
// for the end-of-batch codes (1-byte codes only, <= 255); tasks [ntasks] the
// warp tasks of the vertices of degree > WIDE_BIG_DEG (hubs of degree >
// WIDE_HUB_CHUNK split in tasks of WIDE_HUB_CHUNK edges; hubparts [nhub]
// their task counts); hubacc [nhub] (32-byte aligned), hubcnt [nhub], bar3
// [3] and ctrl zeroed by the caller.
cudaError_t launch_bfs_wide(int code, int n, int nb, const int* rp, const int* ci, const int* tile_base,
                            const int* strip_len, void* D, void* words, int lcap, const int4* tasks, int ntasks,
                            void* hubacc, int* hubcnt, const int* hubparts, int nhub, unsigned long long* bar3,
                            Ctrl* ctrl, long long timeout_ns, int sm_count, int* maxlevel, int* overflow, int* sweeps,
                            cudaStream_t st) {
  if (lcap < 0 || lcap > 255) return cudaErrorInvalidValue;
  const void* fn = (code == CODE_U8) ? (const void*)bfs_wide_kernel<CODE_U8> : (const void*)bfs_wide_kernel<CODE_F32>;
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 512, 0);
  if (e != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  Words4* w4 = reinterpret_cast<Words4*>(words);
  Words4* hacc = reinterpret_cast<Words4*>(hubacc);
  void* args[] = {&n,    &nb,   (void*)&rp, (void*)&ci,  (void*)&tile_base, (void*)&strip_len,
                  &D,    &w4,   &lcap,      (void*)&tasks, &ntasks,         &hacc, &hubcnt, (void*)&hubparts, &nhub,
                  &bar3,
                  &ctrl, &timeout_ns, &maxlevel, &overflow,  &sweeps};
  return cudaLaunchCooperativeKernel(fn, dim3(bps * sm_count), dim3(512), args, 0, st);
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
