// fd_batch_inst.cuh -- instantiation of the batched layout kernel for one
// layout dimension (FD_BATCH_DIM), with its launch-configuration query and
// launcher.  Included once by each fd_batch_d{1,2,3}.cu.
#include "fd_batch.cuh"

#ifndef FD_BATCH_DIM
#error "FD_BATCH_DIM must be defined"
#endif

#define FD_CAT2(a, b) a##b
#define FD_CAT(a, b) FD_CAT2(a, b)

namespace fdl {

template <int W, int T>
static cudaError_t bconfig_one(int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem) {
  *smem = (size_t)BSmem<FD_BATCH_DIM>::bytes(lut_bytes, n_pad_max, W, nbuf);
  cudaError_t e = cudaFuncSetAttribute(fd_batch_kernel<FD_BATCH_DIM, W, T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fd_batch_kernel<FD_BATCH_DIM, W, T>, BGT * W,
                                                       *smem);
}

// Resident CTAs per SM of the launch shape: the least over the three tile
// edges (every class runs at the same grid and shared-memory size).
template <int W>
static cudaError_t bconfig_w(int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem) {
  int b0 = 0, b1 = 0, b2 = 0;
  cudaError_t e = bconfig_one<W, TILE>(lut_bytes, n_pad_max, nbuf, &b0, smem);
  if (e == cudaSuccess) e = bconfig_one<W, 64>(lut_bytes, n_pad_max, nbuf, &b1, smem);
  if (e == cudaSuccess) e = bconfig_one<W, 32>(lut_bytes, n_pad_max, nbuf, &b2, smem);
  *blocks_per_sm = (b0 < b1) ? ((b0 < b2) ? b0 : b2) : ((b1 < b2) ? b1 : b2);
  return e;
}

cudaError_t FD_CAT(batch_config_d, FD_BATCH_DIM)(int W, int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm,
                                                 size_t* smem) {
  return (W == 1) ? bconfig_w<1>(lut_bytes, n_pad_max, nbuf, blocks_per_sm, smem)
                  : bconfig_w<2>(lut_bytes, n_pad_max, nbuf, blocks_per_sm, smem);
}

// Launches the persistent kernel of tile class cls (0: T = 128, 1: 64, 2: 32).
cudaError_t FD_CAT(launch_batch_d, FD_BATCH_DIM)(int W, int cls, const BParams* p, int grid, size_t smem,
                                                 cudaStream_t st) {
  if (W == 1) {
    if (cls == 0) fd_batch_kernel<FD_BATCH_DIM, 1, TILE><<<grid, BGT, smem, st>>>(p);
    else if (cls == 1) fd_batch_kernel<FD_BATCH_DIM, 1, 64><<<grid, BGT, smem, st>>>(p);
    else fd_batch_kernel<FD_BATCH_DIM, 1, 32><<<grid, BGT, smem, st>>>(p);
  } else {
    if (cls == 0) fd_batch_kernel<FD_BATCH_DIM, 2, TILE><<<grid, 2 * BGT, smem, st>>>(p);
    else if (cls == 1) fd_batch_kernel<FD_BATCH_DIM, 2, 64><<<grid, 2 * BGT, smem, st>>>(p);
    else fd_batch_kernel<FD_BATCH_DIM, 2, 32><<<grid, 2 * BGT, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace fdl
