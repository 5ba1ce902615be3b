// The FP64 fused multiply-add rate of the current GPU (the denominator of the
// FP64 path's compute roofline), measured with CUDA events: every thread runs
// eight independent FMA chains (enough to cover the pipeline latency).
#include <cuda_runtime.h>

#include "nupm_internal.h"

namespace nupm {
namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fp64_fma(int iters, double b, double c, double* out) {
  double v[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) v[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) v[k] = fma(v[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += v[k];
  if (s == 12345.678) out[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace nupm

using namespace nupm;

extern "C" int pm_measure_fp64_fma(int32_t iters, double* tflops, void* cuda_stream) {
  if (!tflops || iters < 1) return PM_ERR_INVALID;
  *tflops = 0.0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kPeakThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  k_fp64_fma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.9999999, 1e-7, nullptr);   // warm-up
  cudaEventRecord(e0, s);
  k_fp64_fma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.9999999, 1e-7, nullptr);
  cudaEventRecord(e1, s);
  float ms = 0.0f;
  const cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.0f)) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  const double flops = 2.0 * kPeakChains * 16.0 * (double)iters * blocks * kPeakThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return PM_OK;
}
