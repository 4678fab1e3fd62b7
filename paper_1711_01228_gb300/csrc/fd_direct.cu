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
// identity), and inverted in place by blocked Gauss-Jordan elimination
// without pivoting (stable for a positive definite matrix), 128 x 128
// blocks.  Step k:
//     P      = (M_kk)^-1                 one CTA, unblocked, in shared memory
//     M_kj  := P M_kj          (j != k)  row panel
//     M_ij  -= M_ik M_kj    (i, j != k)  trailing update (old M_ik, new M_kj)
//     M_ik  := -M_ik P         (i != k)  column panel
//     M_kk  := P
// which leaves A'^-1 after the last step.  The three multiplications share
// one 128 x 128 x 128 FP32 block product from shared memory (8 x 8 outputs
// per thread).
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_internal.cuh"

namespace fdl {

namespace {

constexpr int NB = TILE;       // block side of the elimination
constexpr int LDT = NB + 4;    // shared-memory row stride (floats): 16-byte rows, fewer bank conflicts
constexpr int MM_THREADS = 256;
constexpr size_t MM_SMEM = 2 * (size_t)NB * LDT * sizeof(float);

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
      float d;
      if (code == CODE_U8) d = (float)reinterpret_cast<const unsigned char*>(D)[(size_t)t * TILE * TILE + off];
      else d = reinterpret_cast<const float*>(D)[(size_t)t * TILE * TILE + off];
      sd[jl * SL + il] = d;
    }
    __syncthreads();
    // entry (i, j) of A': s_i + shift on the diagonal, -d_ij^-2 + shift off it;
    // the identity on the padding
    auto value = [&](int i, int j, float d) -> float {
      if (i >= n || j >= n) return (i == j) ? 1.f : 0.f;
      if (i == j) return s[i] + shift;
      const float w = (d > 0.f) ? 1.f / (d * d) : 0.f;
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
// Loads the 128 x 128 block at g (leading dimension ld) into shared memory,
// row-major (dst[r][c]) or transposed (dst[c][r]).
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

// acc[q][u] += sum_k A[own(ty,q)][k] * B[k][own(tx,u)], with At = A transposed
// and Bs = B, both [NB][LDT] in shared memory.
__device__ __forceinline__ void block_mma(const float* At, const float* Bs, float (&acc)[8][8], int ty, int tx) {
#pragma unroll 2
  for (int k = 0; k < NB; ++k) {
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

__device__ __forceinline__ void store_acc(float* g, size_t ld, const float (&acc)[8][8], int ty, int tx, float scale) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float* row = g + (size_t)own(ty, q) * ld;
    *reinterpret_cast<float4*>(row + 4 * tx) =
        make_float4(scale * acc[q][0], scale * acc[q][1], scale * acc[q][2], scale * acc[q][3]);
    *reinterpret_cast<float4*>(row + 64 + 4 * tx) =
        make_float4(scale * acc[q][4], scale * acc[q][5], scale * acc[q][6], scale * acc[q][7]);
  }
}

// ------------------------------------------------------------ elimination
// P = (M_kk)^-1 by unblocked Gauss-Jordan in shared memory; M_kk := P.  A
// pivot that is not positive (impossible for a positive definite matrix in
// exact arithmetic) sets *err and is replaced by 1 so that the step ends.
__global__ void __launch_bounds__(512) gj_pivot_kernel(float* __restrict__ M, size_t ld, int k, float* __restrict__ P,
                                                       int* err) {
  extern __shared__ __align__(16) float S[];  // [NB][LDT]
  float* g = M + (size_t)k * NB * ld + (size_t)k * NB;
  load_block(S, g, ld, false);
  __syncthreads();
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int p = 0; p < NB; ++p) {
    float piv = S[p * LDT + p];
    if (!(piv > 0.f) || !isfinite(piv)) {
      if (tid == 0) atomicExch(err, 1);
      piv = 1.f;
    }
    const float inv = 1.f / piv;
    for (int j = tid; j < NB; j += nt)
      if (j != p) S[p * LDT + j] *= inv;
    __syncthreads();
    for (int e = tid; e < NB * NB; e += nt) {
      const int i = e / NB, j = e % NB;
      if (i != p && j != p) S[i * LDT + j] = fmaf(-S[i * LDT + p], S[p * LDT + j], S[i * LDT + j]);
    }
    __syncthreads();
    for (int i = tid; i < NB; i += nt) S[i * LDT + p] = (i == p) ? inv : -S[i * LDT + p] * inv;
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += nt) {
    const int i = e / NB, j = e % NB;
    P[i * NB + j] = S[i * LDT + j];
    g[(size_t)i * ld + j] = S[i * LDT + j];
  }
}

// Row panel: M_kj := P M_kj for the nb - 1 blocks j != k.
__global__ void __launch_bounds__(MM_THREADS) gj_row_kernel(float* __restrict__ M, size_t ld, int k,
                                                            const float* __restrict__ P) {
  extern __shared__ __align__(16) float sm[];
  float *At = sm, *Bs = sm + NB * LDT;
  const int j = blockIdx.x + (blockIdx.x >= k ? 1 : 0);
  float* g = M + (size_t)k * NB * ld + (size_t)j * NB;
  load_block(At, P, NB, true);
  load_block(Bs, g, ld, false);
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float acc[8][8] = {};
  block_mma(At, Bs, acc, ty, tx);
  store_acc(g, ld, acc, ty, tx, 1.f);
}

// Trailing update: M_ij -= M_ik M_kj for i, j != k.
__global__ void __launch_bounds__(MM_THREADS) gj_update_kernel(float* __restrict__ M, size_t ld, int k, int nb) {
  extern __shared__ __align__(16) float sm[];
  float *At = sm, *Bs = sm + NB * LDT;
  const int m = nb - 1;
  const int ii = blockIdx.x / m, jj = blockIdx.x % m;
  const int i = ii + (ii >= k ? 1 : 0), j = jj + (jj >= k ? 1 : 0);
  load_block(At, M + (size_t)i * NB * ld + (size_t)k * NB, ld, true);
  load_block(Bs, M + (size_t)k * NB * ld + (size_t)j * NB, ld, false);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float* g = M + (size_t)i * NB * ld + (size_t)j * NB;
  float acc[8][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float* row = g + (size_t)own(ty, q) * ld;
    const float4 c0 = *reinterpret_cast<const float4*>(row + 4 * tx);
    const float4 c1 = *reinterpret_cast<const float4*>(row + 64 + 4 * tx);
    // negated, so that the shared product adds: -(M_ij - M_ik M_kj) = -M_ij + M_ik M_kj
    acc[q][0] = -c0.x, acc[q][1] = -c0.y, acc[q][2] = -c0.z, acc[q][3] = -c0.w;
    acc[q][4] = -c1.x, acc[q][5] = -c1.y, acc[q][6] = -c1.z, acc[q][7] = -c1.w;
  }
  __syncthreads();
  block_mma(At, Bs, acc, ty, tx);
  store_acc(g, ld, acc, ty, tx, -1.f);
}

// Column panel: M_ik := -M_ik P for the nb - 1 blocks i != k.
__global__ void __launch_bounds__(MM_THREADS) gj_col_kernel(float* __restrict__ M, size_t ld, int k,
                                                            const float* __restrict__ P) {
  extern __shared__ __align__(16) float sm[];
  float *At = sm, *Bs = sm + NB * LDT;
  const int i = blockIdx.x + (blockIdx.x >= k ? 1 : 0);
  float* g = M + (size_t)i * NB * ld + (size_t)k * NB;
  load_block(At, g, ld, true);
  load_block(Bs, P, NB, false);
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float acc[8][8] = {};
  block_mma(At, Bs, acc, ty, tx);
  store_acc(g, ld, acc, ty, tx, -1.f);
}

}  // namespace

// Builds A' from the distance tiles and inverts it in place (stream-ordered;
// *err is set on the device if a pivot was not positive).
cudaError_t launch_direct_factor(int n, int n_pad, int nb, int code, const void* D, const int2* tile_ik, int ntiles,
                                 const float* s, float shift, float* M, float* P, int* err, int sm_count,
                                 cudaStream_t st) {
  const size_t build_smem = (size_t)TILE * (TILE + 1) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(dense_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gj_pivot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(NB * LDT * 4));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gj_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MM_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MM_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gj_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MM_SMEM);
  if (e != cudaSuccess) return e;
  const int bgrid = ntiles < 4 * sm_count ? ntiles : 4 * sm_count;
  dense_build_kernel<<<bgrid, 256, build_smem, st>>>(n, n_pad, nb, code, D, tile_ik, ntiles, s, shift, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ld = (size_t)n_pad;
  for (int k = 0; k < nb; ++k) {
    gj_pivot_kernel<<<1, 512, NB * LDT * 4, st>>>(M, ld, k, P, err);
    if (nb > 1) {
      gj_row_kernel<<<nb - 1, MM_THREADS, MM_SMEM, st>>>(M, ld, k, P);
      gj_update_kernel<<<(unsigned)((nb - 1) * (nb - 1)), MM_THREADS, MM_SMEM, st>>>(M, ld, k, nb);
      gj_col_kernel<<<nb - 1, MM_THREADS, MM_SMEM, st>>>(M, ld, k, P);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fdl
