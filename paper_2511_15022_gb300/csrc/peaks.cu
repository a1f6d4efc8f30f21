// peaks.cu -- FP32 FMA and MUFU (special-function unit) throughput microbenchmarks: the
// denominators of the arithmetic rooflines the benchmark reports beside the HBM one.
//
// Each thread runs 8 independent dependency chains so that the pipes, not latency, limit
// the rate; the grid is 8 CTAs of 256 threads per SM.  The results are written out only
// under a condition that never holds (and to a NULL sink, so never at all), which keeps the
// chains from being removed as dead code.
#include <cuda_runtime.h>

#include "cgh_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1234.5f && out) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float v) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// x <- 2^-x stays inside (0.5, 1]: one MUFU operation per step, the negation is an operand
// modifier
__global__ void __launch_bounds__(256) k_sfu_peak(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x % 7 + c) * 0.1f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = ex2_approx(-x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1234.5f && out) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class F>
cgh_status time_ms(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cgh_record_error(CGH_ERR_CUDA, "cgh_measure_peaks: event creation failed");
  launch();  // warm-up
  cudaEventRecord(e0, s);
  launch();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" cgh_status cgh_measure_peaks(double* fp32_flops_per_s, double* sfu_ops_per_s,
                                        void* stream) {
  if (!fp32_flops_per_s || !sfu_ops_per_s)
    return cgh_record_error(CGH_ERR_ARG, "cgh_measure_peaks: NULL output");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * 8, threads = 256;
  float* sink = nullptr;  // never written (see the kernels)
  const int fma_iters = 16384, sfu_iters = 2048;
  float ms = 0.f;
  cgh_status st = time_ms([&] { k_fma_peak<<<blocks, threads, 0, s>>>(sink, fma_iters, 0.999f, 1e-3f); }, s, &ms);
  if (st != CGH_OK) return st;
  *fp32_flops_per_s = 2.0 * kChains * 4.0 * fma_iters * (double)blocks * threads / (ms * 1e-3);
  st = time_ms([&] { k_sfu_peak<<<blocks, threads, 0, s>>>(sink, sfu_iters); }, s, &ms);
  if (st != CGH_OK) return st;
  *sfu_ops_per_s = (double)kChains * 4.0 * sfu_iters * (double)blocks * threads / (ms * 1e-3);
  return CGH_OK;
}
