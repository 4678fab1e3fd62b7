// fd_noalloc.cu -- stress evaluation that allocates no memory.
//
// fd_energy_noalloc() computes the same stress as fd_energy(), but from a
// caller-supplied dense distance matrix and without creating a handle.  Its
// only scratch is the file-scope device array below, so it never calls
// cudaMalloc, cudaFree or any allocating library routine.  It exists for
// callers that cannot allocate device memory: code running inside a process
// whose GPU memory is owned by another allocator (a framework's caching
// allocator or a fixed arena), where an extra cudaMalloc can fail or force a
// device-wide synchronisation, and latency-critical loops that must not pay
// for an allocation.
//
// Sharing rules (see include/fd_layout.h): every call on a device uses the
// same scratch array, so calls whose kernels overlap on the GPU (different
// streams, or host threads racing) corrupt each other's partial sums.  The
// array keeps the previous call's contents; every slot a call reads is first
// written by that same call.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_layout.h"

namespace {

constexpr int NA_THREADS = 128;
constexpr int NA_MAX_BLOCKS = FD_NOALLOC_MAX_N / NA_THREADS;

// Per-block partial stresses, then the final sum in the last slot.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 1];

__device__ __forceinline__ float na_kahan(float& s, float& c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
  return s;
}

// Thread i sums w_ij (||x_i - x_j|| - d_ij)^2 over j > i (Eq. (1)), reading
// d_ij from the strictly lower triangle D[j * n + i] so that a warp's loads
// are contiguous.  A pair with d_ij <= 0 is no pair (weight 0), as a zero
// code is in fd_energy's distance tiles.  Block partials are FP64, summed in
// a fixed order.
__global__ void __launch_bounds__(NA_THREADS) na_stress_partials(const float* __restrict__ X,
                                                                 const float* __restrict__ D, int n, int dim,
                                                                 double* partials) {
  __shared__ double red[NA_THREADS];
  const int i = blockIdx.x * NA_THREADS + threadIdx.x;
  float s = 0.f, c = 0.f;
  if (i < n) {
    float xi[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < dim; ++d) xi[d] = X[(size_t)i * dim + d];
    for (int j = i + 1; j < n; ++j) {
      float r2 = 0.f;
      for (int d = 0; d < dim; ++d) {
        const float t = xi[d] - X[(size_t)j * dim + d];
        r2 = fmaf(t, t, r2);
      }
      const float dij = D[(size_t)j * n + i];
      if (!(dij > 0.f)) continue;
      const float e = sqrtf(r2) - dij;
      na_kahan(s, c, e * e / (dij * dij));
    }
  }
  red[threadIdx.x] = (double)s - (double)c;
  __syncthreads();
  for (int k = NA_THREADS / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(NA_THREADS) na_stress_final(const double* partials, int nblocks, double* out) {
  __shared__ double red[NA_THREADS];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) v += partials[b];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int k = NA_THREADS / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// 1: device memory of device `dev` (or managed memory, reachable from every
// device); 0: host memory, another device's memory, or not a CUDA pointer.
int na_on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeManaged) return 1;
  return (a.type == cudaMemoryTypeDevice && a.device == dev) ? 1 : 0;
}

// Device address of the scratch array in the current device's context.  The
// address is looked up on every call (a host-side lookup that allocates
// nothing): after cudaDeviceReset, or anything else that recreates the
// context, the library's device image is loaded again and the array may sit
// elsewhere, so a cached address could point at freed memory.
fd_status na_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return FD_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return FD_OK;
}

}  // namespace

extern "C" fd_status fd_energy_noalloc(const float* X, const float* D, int32_t n, int32_t dim, double* f_out,
                                       void* cuda_stream) {
  if (!X || !D || !f_out || n < 1 || dim < 1 || dim > 3) return FD_ERR_ARG;
  if (n > FD_NOALLOC_MAX_N) return FD_ERR_ARG;  // more blocks than the scratch array holds
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FD_ERR_CUDA;
  }
  // X and D must be reachable by the kernels on the current device
  if (!na_on_device(X, dev) || !na_on_device(D, dev)) return FD_ERR_ARG;
  double* scratch = nullptr;
  fd_status s = na_scratch(&scratch);
  if (s != FD_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nblocks = (n + NA_THREADS - 1) / NA_THREADS;
  // a device f_out is written by the kernel; anything else (host memory, or
  // another device's memory) gets the value copied from the scratch array
  const bool dev_out = na_on_device(f_out, dev) != 0;
  double* result = dev_out ? f_out : scratch + NA_MAX_BLOCKS;
  na_stress_partials<<<nblocks, NA_THREADS, 0, st>>>(X, D, n, dim, scratch);
  na_stress_final<<<1, NA_THREADS, 0, st>>>(scratch, nblocks, result);
  // the value is also read back to the stack to check it is finite
  double f = 0.0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, result, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FD_ERR_CUDA;
  }
  if (!dev_out) *f_out = f;
  if (!(f == f && f - f == 0.0)) return FD_ERR_NONFINITE;
  return FD_OK;
}
