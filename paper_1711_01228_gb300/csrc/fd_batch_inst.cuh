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

template <int W>
static cudaError_t bconfig_one(int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem) {
  *smem = (size_t)BSmem<FD_BATCH_DIM>::bytes(lut_bytes, n_pad_max, W, nbuf);
  cudaError_t e = cudaFuncSetAttribute(fd_batch_kernel<FD_BATCH_DIM, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)*smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fd_batch_kernel<FD_BATCH_DIM, W>, BGT * W,
                                                       *smem);
}

cudaError_t FD_CAT(batch_config_d, FD_BATCH_DIM)(int W, int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm,
                                                 size_t* smem) {
  return (W == 1) ? bconfig_one<1>(lut_bytes, n_pad_max, nbuf, blocks_per_sm, smem)
                  : bconfig_one<2>(lut_bytes, n_pad_max, nbuf, blocks_per_sm, smem);
}

cudaError_t FD_CAT(launch_batch_d, FD_BATCH_DIM)(int W, const BParams* p, int grid, size_t smem, cudaStream_t st) {
  if (W == 1)
    fd_batch_kernel<FD_BATCH_DIM, 1><<<grid, BGT, smem, st>>>(p);
  else
    fd_batch_kernel<FD_BATCH_DIM, 2><<<grid, 2 * BGT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace fdl
