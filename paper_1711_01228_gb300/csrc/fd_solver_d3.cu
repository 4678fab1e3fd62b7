// fd_solver_d3.cu -- instantiation of the cooperative layout kernel for
// dim = 3 (one translation unit per dimension so that they build in parallel).
#include "fd_solver.cuh"

namespace fdl {

template <int CODE>
static cudaError_t config_one(size_t lut_bytes, int nbuf, int tps, int* blocks_per_sm, size_t* smem) {
  if (tps != 1) return cudaErrorInvalidValue;  // one tile per stage in 3-D
  using L = SmemLayout<3, CODE>;
  *smem = (size_t)L::bytes(nbuf, CODE == CODE_U8 ? (int)lut_bytes : 0, tps);
  cudaError_t e = cudaFuncSetAttribute(fd_main_kernel<3, CODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)*smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fd_main_kernel<3, CODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  int b0 = 0, b1 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, fd_main_kernel<3, CODE, false>, CTA, *smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, fd_main_kernel<3, CODE, true>, CTA, *smem);
  *blocks_per_sm = b0 < b1 ? b0 : b1;
  return e;
}

cudaError_t main_config_d3(int code, size_t lut_bytes, int nbuf, int tps, int* blocks_per_sm, size_t* smem) {
  return code == CODE_U8 ? config_one<CODE_U8>(lut_bytes, nbuf, tps, blocks_per_sm, smem)
                         : config_one<CODE_F32>(lut_bytes, nbuf, tps, blocks_per_sm, smem);
}

cudaError_t launch_main_d3(int code, const KParams& p, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<KParams*>(&p)};
  const void* fn;
  if (p.enum_omega)
    fn = (code == CODE_U8) ? (const void*)fd_main_kernel<3, CODE_U8, true> : (const void*)fd_main_kernel<3, CODE_F32, true>;
  else
    fn = (code == CODE_U8) ? (const void*)fd_main_kernel<3, CODE_U8, false>
                           : (const void*)fd_main_kernel<3, CODE_F32, false>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(CTA), args, smem, st);
}

}  // namespace fdl
