// fd_direct.cu -- the direct solver of Eq. (2-5): L^W is fixed over the
// whole run (Sec. 2 lists Cholesky factorisation among the solvers for it),
// so it is inverted once and every H step applies the inverse.
//
// The pinned system (row and column of vertex 0 removed) has a condition
// number about n times that of L^W, too much for FP32.  The inverse here is
// of the shifted matrix
//     A' = L^W + (sigma / n) 1 1^T,   sigma = mean_i s_i,
// which is positive definite with the spectrum of L^W except that the null
// vector 1 gets eigenvalue sigma.  For a right-hand side with zero sum (every
// L^X X has one, and so has every residual of Eq. (2-5)) A'^-1 b solves
// L^W z = b; pinning vertex 0 is then a translation.
//
// A' is stored dense, FP32, n_pad x n_pad (padding rows and columns are the
// identity), and inverted in place by the symmetric sweep (Gauss-Jordan
// elimination that keeps the matrix symmetric; no pivoting, which is stable
// for a positive definite matrix) in 128 x 128 blocks, updating only the
// lower triangle: n_pad^3 flops, half of plain Gauss-Jordan.  The block
// products are FP32 on the CUDA cores, 128 x 128 outputs per CTA (8 x 8 per
// thread) from shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_internal.cuh"

namespace fdl {

namespace {

constexpr int NB = TILE;       // block side of the elimination
constexpr int LDT = NB + 4;    // shared-memory row stride (floats): 16-byte rows, fewer bank conflicts

// ---------------------------------------------------------------- build A'
// One CTA per stored tile (I, J = (I + k) mod nb): its 128 x 128 distances go
// to shared memory, then block (I, J) and its transpose (J, I) of A' are
// written row by row.
__global__ void __launch_bounds__(256) dense_build_kernel(int n, int n_pad, int nb, int code, const void* __restrict__ D,
                                                          const int2* __restrict__ tile_ik, int ntiles,
                                                          const float* __restrict__ s, float shift,
                                                          float* __restrict__ M) {
  extern __shared__ __align__(16) float sd[];  // [TILE][TILE + 1]: sd[jl][il] = d(I*T+il, J*T+jl)
  constexpr int SL = TILE + 1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 ik = tile_ik[t];
    const int I = ik.x, J = (ik.x + ik.y) % nb;
    const bool diag = (ik.y == 0);
    __syncthreads();  // the previous tile's readers are done
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
      const int jl = e / TILE, il = e % TILE;
      // off-diagonal tiles hold pair (il, jl) at jl * TILE + il; the diagonal
      // tile holds it at max * TILE + min
      const int off = diag ? (max(il, jl) * TILE + min(il, jl)) : e;
      // the weight d^-2: from the hop count, or the square of a float tile's 1/d
      float w;
      if (code == CODE_U8) {
        const float d = (float)reinterpret_cast<const unsigned char*>(D)[(size_t)t * TILE * TILE + off];
        w = (d > 0.f) ? 1.f / (d * d) : 0.f;
      } else {
        const float c = reinterpret_cast<const float*>(D)[(size_t)t * TILE * TILE + off];
        w = c * c;
      }
      sd[jl * SL + il] = w;
    }
    __syncthreads();
    // entry (i, j) of A': s_i + shift on the diagonal, -d_ij^-2 + shift off it;
    // the identity on the padding
    auto value = [&](int i, int j, float w) -> float {
      if (i >= n || j >= n) return (i == j) ? 1.f : 0.f;
      if (i == j) return s[i] + shift;
      return shift - w;
    };
    // block (I, J): row i = I*T + il, columns J*T + jl (coalesced over jl)
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
      const int il = e / TILE, jl = e % TILE;
      const int i = I * TILE + il, j = J * TILE + jl;
      M[(size_t)i * n_pad + j] = value(i, j, sd[jl * SL + il]);
    }
    if (!diag) {
      // block (J, I): row j = J*T + jl, columns I*T + il (coalesced over il)
      for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        const int jl = e / TILE, il = e % TILE;
        const int i = I * TILE + il, j = J * TILE + jl;
        M[(size_t)j * n_pad + i] = value(j, i, sd[jl * SL + il]);
      }
    }
  }
}

// ------------------------------------------------------------- block product
// Loads the 128 x 128 block at g (leading dimension ld) into shared memory
// (row stride LDT), row-major (dst[r][c]) or transposed (dst[c][r]).
__device__ __forceinline__ void load_block(float* dst, const float* g, size_t ld, bool transpose) {
  if (!transpose) {
    // a warp reads one row (512 contiguous bytes) and writes it as one row
    for (int e = threadIdx.x; e < NB * NB / 4; e += blockDim.x) {
      const int r = e / (NB / 4), c4 = (e % (NB / 4)) * 4;
      *reinterpret_cast<float4*>(dst + r * LDT + c4) = *reinterpret_cast<const float4*>(g + (size_t)r * ld + c4);
    }
  } else {
    // a warp reads 32 B (a whole sector) of 32 consecutive rows and writes
    // 8 rows of the transpose, each 32 consecutive floats (no bank conflict)
    for (int e = threadIdx.x; e < NB * NB / 8; e += blockDim.x) {
      const int r = e % NB, c8 = (e / NB) * 8;
      const float* src = g + (size_t)r * ld + c8;
      const float4 v0 = *reinterpret_cast<const float4*>(src);
      const float4 v1 = *reinterpret_cast<const float4*>(src + 4);
      const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[(c8 + q) * LDT + r] = v[q];
    }
  }
}

// Thread (ty, tx) of a 16 x 16 arrangement owns rows {4ty..4ty+3, 64+4ty..64+4ty+3}
// and the same columns with tx.
__device__ __forceinline__ int own(int base, int q) { return (q < 4) ? 4 * base + q : 64 + 4 * base + (q - 4); }

// acc[q][u] += sum_{k < K} A[own(ty,q)][k] * B[k][own(tx,u)], with At = A
// transposed and Bs = B, both [K][LDT] in shared memory.
template <int K, int U>
__device__ __forceinline__ void block_mma(const float* At, const float* Bs, float (&acc)[8][8], int ty, int tx) {
#pragma unroll U
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(At + k * LDT + 4 * ty);
    const float4 a1 = *reinterpret_cast<const float4*>(At + k * LDT + 64 + 4 * ty);
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + k * LDT + 4 * tx);
    const float4 b1 = *reinterpret_cast<const float4*>(Bs + k * LDT + 64 + 4 * tx);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[q][u] = fmaf(a[q], b[u], acc[q][u]);
  }
}

// The same product with two-wide FMAs (fma.rn.f32x2: two independent IEEE
// FMAs, so every output is rounded exactly as by fmaf, in the same order):
// acc[q][v] holds columns own(tx, 2v) and own(tx, 2v + 1) of row own(ty, q).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float lo, float hi) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void up2(f2x v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
template <int K, int U>
__device__ __forceinline__ void block_mma2(const float* At, const float* Bs, f2x (&acc)[8][4], int ty, int tx) {
#pragma unroll U
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(At + k * LDT + 4 * ty);
    const float4 a1 = *reinterpret_cast<const float4*>(At + k * LDT + 64 + 4 * ty);
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(Bs + k * LDT + 4 * tx);
    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(Bs + k * LDT + 64 + 4 * tx);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const f2x b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const f2x aa = pk2(a[q], a[q]);
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[q][v] = fma2(aa, b[v], acc[q][v]);
    }
  }
}

__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------------- the sweep
// The symmetric sweep keeps the matrix symmetric, so only blocks (i, j) with
// i >= j are kept up to date.  Step k (P = (M_kk)^-1):
//     M_ij -= (M_ik P) M_kj   (i >= j, i, j != k)   trailing update
//     M_ik := M_ik P          (i != k)              panel
//     M_kk := -P
// After every block has been the pivot, the lower triangle holds -A'^-1.

// P = (M_kk)^-1 by unblocked Gauss-Jordan, the block held in registers:
// thread t owns rows 8 (t / 32) .. + 7 and columns 4 (t % 32) .. + 3.  Per
// pivot p the owners of row p and column p publish them in shared memory
// (two buffers, alternating, so one barrier per pivot).  Writes P to Pbuf
// and -P to M_kk.  A pivot that is not positive (impossible for a positive
// definite matrix in exact arithmetic) sets *err and is replaced by 1.
constexpr int PIV_THREADS = 512;
__global__ void __launch_bounds__(PIV_THREADS) sw_pivot_kernel(float* __restrict__ M, size_t ld, int k,
                                                                float* __restrict__ P, int* err) {
  __shared__ float rowb[2][NB], colb[2][NB];
  const int t = threadIdx.x, r0 = (t / 32) * 8, c0 = (t % 32) * 4;
  float* g = M + (size_t)k * NB * ld + (size_t)k * NB;
  float a[8][4];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = *reinterpret_cast<const float4*>(g + (size_t)(r0 + q) * ld + c0);
    a[q][0] = v.x, a[q][1] = v.y, a[q][2] = v.z, a[q][3] = v.w;
  }
  bool bad = false;
  for (int p = 0; p < NB; ++p) {
    const int b = p & 1;
    if (p >= r0 && p < r0 + 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (r0 + q == p)
#pragma unroll
          for (int u = 0; u < 4; ++u) rowb[b][c0 + u] = a[q][u];
    }
    if (p >= c0 && p < c0 + 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u == p)
#pragma unroll
          for (int q = 0; q < 8; ++q) colb[b][r0 + q] = a[q][u];
    }
    __syncthreads();
    float piv = rowb[b][p];
    if (!(piv > 0.f) || !isfinite(piv)) {
      bad = true;
      piv = 1.f;
    }
    const float inv = 1.f / piv;
    float rj[4], ci[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) rj[u] = rowb[b][c0 + u];
#pragma unroll
    for (int q = 0; q < 8; ++q) ci[q] = colb[b][r0 + q] * inv;
    // a_ij - a_ip a_pj / piv for every entry; row p and column p are then
    // overwritten by their owners (warp-uniform for the row, one lane per
    // warp for the column)
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) a[q][u] = fmaf(-ci[q], rj[u], a[q][u]);
    if (p >= r0 && p < r0 + 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (r0 + q == p)
#pragma unroll
          for (int u = 0; u < 4; ++u) a[q][u] = rj[u] * inv;  // row p scaled
    }
    if (p >= c0 && p < c0 + 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u == p)
#pragma unroll
          for (int q = 0; q < 8; ++q) a[q][u] = (r0 + q == p) ? inv : -ci[q];  // column p: -a_ip / piv; pivot 1/piv
    }
  }
  if (bad) atomicExch(err, 1);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    *reinterpret_cast<float4*>(P + (r0 + q) * NB + c0) = make_float4(a[q][0], a[q][1], a[q][2], a[q][3]);
    *reinterpret_cast<float4*>(g + (size_t)(r0 + q) * ld + c0) = make_float4(-a[q][0], -a[q][1], -a[q][2], -a[q][3]);
  }
}

// Panel, one CTA per block i != k: Q_i = M_ik P with M_ik read from the
// lower triangle (block (i, k) if i > k, the transpose of block (k, i) if
// i < k).  Writes the update's two operands, both [K][row] so that its
// copies are plain: QT_i = Q_i^T and AT_i = M_ik^T (before scaling); and
// the new panel M_ik := Q_i into the lower triangle.
constexpr int MM_THREADS = 256;
constexpr size_t PANEL_SMEM = 2 * (size_t)NB * LDT * sizeof(float);
__global__ void __launch_bounds__(MM_THREADS) sw_panel_kernel(float* __restrict__ M, size_t ld, int k,
                                                              const float* __restrict__ P, float* __restrict__ QT,
                                                              float* __restrict__ AT) {
  extern __shared__ __align__(16) float sm[];
  float *At = sm, *Bs = sm + NB * LDT;
  const int i = blockIdx.x + (blockIdx.x >= k ? 1 : 0);
  const bool below = i > k;
  float* gpan = below ? M + (size_t)i * NB * ld + (size_t)k * NB : M + (size_t)k * NB * ld + (size_t)i * NB;
  load_block(At, gpan, ld, below);  // At[kk][r] = M_ik[r][kk]
  load_block(Bs, P, NB, false);
  __syncthreads();
  float* at = AT + (size_t)i * NB * NB;
  for (int e = threadIdx.x; e < NB * NB / 4; e += blockDim.x) {
    const int r = e / (NB / 4), c4 = (e % (NB / 4)) * 4;
    *reinterpret_cast<float4*>(at + r * NB + c4) = *reinterpret_cast<const float4*>(At + r * LDT + c4);
  }
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float acc[8][8] = {};
  block_mma<NB, 2>(At, Bs, acc, ty, tx);
  __syncthreads();  // At is reused for Q_i
  constexpr int LQ = NB + 1;
  float* Cs = sm;  // [NB][LQ]: Cs[r][c] = Q_i[r][c]
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int u = 0; u < 8; ++u) Cs[own(ty, q) * LQ + own(tx, u)] = acc[q][u];
  __syncthreads();
  float* qt = QT + (size_t)i * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int a = e / NB, b = e % NB;  // QT_i[a][b] = Q_i[b][a]
    const float v = Cs[b * LQ + a];
    qt[a * NB + b] = v;
    if (!below) gpan[(size_t)a * ld + b] = v;  // block (k, i) = Q_i^T
  }
  if (below)
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, c = e % NB;
      gpan[(size_t)r * ld + c] = Cs[r * LQ + c];  // block (i, k) = Q_i
    }
}

// Trailing update of the lower blocks: one CTA per block (i, j), i >= j,
// i, j != k:  M_ij -= Q_i M_kj = sum_kk QT_i[kk][r] AT_j[kk][c].  The two
// operands stream through shared memory in chunks of BK rows, two stages,
// by cp.async; the output block stays in registers.  Two CTAs per SM.
constexpr int BK = 32;
constexpr size_t UPD_STAGE = 2 * (size_t)BK * LDT;  // floats per stage (QT chunk + AT chunk)
constexpr size_t UPD_SMEM = 2 * UPD_STAGE * sizeof(float);
__global__ void __launch_bounds__(MM_THREADS, 2) sw_update_kernel(float* __restrict__ M, size_t ld, int k, int nb,
                                                                 const float* __restrict__ QT,
                                                                 const float* __restrict__ AT) {
  extern __shared__ __align__(16) float sm[];
  // block b of the lower triangle of an m x m grid, row-major: ii (ii + 1) / 2 <= b
  const int b = blockIdx.x;
  int ii = (int)((sqrtf(8.f * b + 1.f) - 1.f) * 0.5f);
  while ((ii + 1) * (ii + 2) / 2 <= b) ++ii;
  while (ii * (ii + 1) / 2 > b) --ii;
  const int jj = b - ii * (ii + 1) / 2;
  const int i = ii + (ii >= k ? 1 : 0), j = jj + (jj >= k ? 1 : 0);
  const float* qa = QT + (size_t)i * NB * NB;
  const float* ab = AT + (size_t)j * NB * NB;
  auto issue = [&](int chunk, int stage) {
    float* As = sm + stage * UPD_STAGE;
    float* Bs = As + BK * LDT;
    for (int e = threadIdx.x; e < BK * NB / 4; e += blockDim.x) {
      const int r = e / (NB / 4), c4 = (e % (NB / 4)) * 4;
      cp_async16(As + r * LDT + c4, qa + (size_t)(chunk * BK + r) * NB + c4);
      cp_async16(Bs + r * LDT + c4, ab + (size_t)(chunk * BK + r) * NB + c4);
    }
    cp_async_commit();
  };
  issue(0, 0);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float* g = M + (size_t)i * NB * ld + (size_t)j * NB;
  f2x acc[8][4];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float* row = g + (size_t)own(ty, q) * ld;
    const float4 c0 = *reinterpret_cast<const float4*>(row + 4 * tx);
    const float4 c1 = *reinterpret_cast<const float4*>(row + 64 + 4 * tx);
    // negated, so that the block product adds: -(M_ij - Q_i M_kj) = -M_ij + Q_i M_kj
    acc[q][0] = pk2(-c0.x, -c0.y), acc[q][1] = pk2(-c0.z, -c0.w);
    acc[q][2] = pk2(-c1.x, -c1.y), acc[q][3] = pk2(-c1.z, -c1.w);
  }
  constexpr int NCH = NB / BK;
#pragma unroll 1
  for (int c = 0; c < NCH; ++c) {
    if (c + 1 < NCH) {
      issue(c + 1, (c + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // chunk c visible to every thread
    const float* As = sm + (c & 1) * UPD_STAGE;
    block_mma2<BK, 2>(As, As + BK * LDT, acc, ty, tx);
    __syncthreads();  // every thread is done with the stage before chunk c + 2 overwrites it
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float v[8];
#pragma unroll
    for (int w = 0; w < 4; ++w) up2(acc[q][w], v[2 * w], v[2 * w + 1]);
    float* row = g + (size_t)own(ty, q) * ld;
    *reinterpret_cast<float4*>(row + 4 * tx) = make_float4(-v[0], -v[1], -v[2], -v[3]);
    *reinterpret_cast<float4*>(row + 64 + 4 * tx) = make_float4(-v[4], -v[5], -v[6], -v[7]);
  }
}

// Lower triangle holds -A'^-1: negate it and mirror it to the upper
// triangle.  One CTA per lower block (i, j); the transpose goes through
// shared memory so that both writes are row by row.
constexpr size_t FIN_SMEM = (size_t)NB * (NB + 1) * sizeof(float);
__global__ void __launch_bounds__(256) sw_finish_kernel(float* __restrict__ M, size_t ld) {
  extern __shared__ __align__(16) float fin[];
  auto Cs = reinterpret_cast<float(*)[NB + 1]>(fin);
  const int b = blockIdx.x;
  int i = (int)((sqrtf(8.f * b + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= b) ++i;
  while (i * (i + 1) / 2 > b) --i;
  const int j = b - i * (i + 1) / 2;
  float* g = M + (size_t)i * NB * ld + (size_t)j * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    const float v = -g[(size_t)r * ld + c];
    Cs[r][c] = v;
    g[(size_t)r * ld + c] = v;
  }
  if (i == j) return;
  __syncthreads();
  float* h = M + (size_t)j * NB * ld + (size_t)i * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    h[(size_t)r * ld + c] = Cs[c][r];
  }
}

}  // namespace

// Builds A' from the distance tiles and inverts it in place by the
// symmetric sweep (stream-ordered; *err is set on the device if a pivot was
// not positive).  Scratch: P [NB][NB], QT and AT [nb][NB][NB] each.
cudaError_t launch_direct_factor(int n, int n_pad, int nb, int code, const void* D, const int2* tile_ik, int ntiles,
                                 const float* s, float shift, float* M, float* P, float* QT, float* AT, int* err,
                                 int sm_count, cudaStream_t st) {
  const size_t build_smem = (size_t)TILE * (TILE + 1) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(dense_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sw_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sw_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UPD_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sw_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FIN_SMEM);
  if (e != cudaSuccess) return e;
  const int bgrid = ntiles < 4 * sm_count ? ntiles : 4 * sm_count;
  dense_build_kernel<<<bgrid, 256, build_smem, st>>>(n, n_pad, nb, code, D, tile_ik, ntiles, s, shift, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ld = (size_t)n_pad;
  const int m = nb - 1;
  for (int k = 0; k < nb; ++k) {
    sw_pivot_kernel<<<1, PIV_THREADS, 0, st>>>(M, ld, k, P, err);
    if (m > 0) {
      sw_panel_kernel<<<m, MM_THREADS, PANEL_SMEM, st>>>(M, ld, k, P, QT, AT);
      sw_update_kernel<<<(unsigned)(m * (m + 1) / 2), MM_THREADS, UPD_SMEM, st>>>(M, ld, k, nb, QT, AT);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  sw_finish_kernel<<<(unsigned)(nb * (nb + 1) / 2), 256, FIN_SMEM, st>>>(M, ld);
  return cudaGetLastError();
}

}  // namespace fdl
