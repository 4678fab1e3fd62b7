// fd_peak.cu -- FP32 FMA throughput of the device (the denominator of the
// layout kernel's roofline): independent FMA chains in every thread, scalar
// (fma.rn.f32) or packed two-wide (fma.rn.f32x2, the instruction the pair
// passes use), timed with CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_internal.cuh"

namespace fdl {

namespace {

constexpr int CHAINS = 16;  // independent FP32 accumulators per thread

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}

__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <bool PACKED>
__global__ void __launch_bounds__(256) ffma_peak_kernel(float* out, int iters, float a, float b) {
  float acc = 0.f;
  if constexpr (PACKED) {
    unsigned long long x[CHAINS / 2];
    const unsigned long long A = pack2(a, a), B = pack2(b, b);
#pragma unroll
    for (int k = 0; k < CHAINS / 2; ++k) x[k] = pack2(1e-3f * threadIdx.x + k, 0.5f * k);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < CHAINS / 2; ++k) x[k] = fma_x2(x[k], A, B);
#pragma unroll
    for (int k = 0; k < CHAINS / 2; ++k) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
      acc += lo + hi;
    }
  } else {
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = 1e-3f * threadIdx.x + k;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[k]) : "f"(a), "f"(b));
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc += x[k];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

// Best of `reps` timed launches (after one warm-up) of sm_count * 4 CTAs of
// 256 threads; flops = 2 * CHAINS * iters per thread.
cudaError_t measure_fp32_peak(int packed, int sm_count, int reps, double* tflops, double* best_ms) {
  const int grid = sm_count * 4, threads = 256, iters = 1 << 15;
  float* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)grid * threads * sizeof(float));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0);
    if (packed) ffma_peak_kernel<true><<<grid, threads>>>(out, iters, 0.999f, 1e-3f);
    else ffma_peak_kernel<false><<<grid, threads>>>(out, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * CHAINS * (double)iters * grid * threads;
  *best_ms = best;
  *tflops = flops / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace fdl
