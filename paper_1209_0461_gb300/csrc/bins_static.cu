// pm_bin_power_static: binned power spectrum of a caller-owned half spectrum
// (numpy rfftn layout) that allocates no device memory.
//
// Who needs it: codes that reserve all device memory up front in their own
// pool, or that must not allocate inside their time-step loop (a device
// allocation can synchronise the GPU and can fail mid-run), still want the
// P(k) diagnostic of the kick.  The per-block partial sums this reduction
// needs live in a fixed file-scope device array instead of cudaMalloc'd
// memory; the bin thresholds travel as a kernel argument.
//
// Limits: n_kbins <= kStaticMaxBins, ngrid a power of two in [16, 1024].
// The scratch (kStaticBlocks x 3 x kStaticMaxBins doubles, 1.8 MB) is held by
// every device that loads the library, until the process exits.  All calls
// on a device share it and it keeps the last call's contents; every call
// rewrites all of the partials it reads, so nothing must be cleared, but two
// calls that overlap on the GPU (different streams, no ordering) race.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "fft.cuh"
#include "nupm_internal.h"

namespace nupm {
namespace {

constexpr int kStaticMaxBins = 256;
constexpr int kStaticBlocks = 304;   // 2 CTAs per SM of a 152-SM part
constexpr int kStaticWarps = 4;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_bin_scratch[(size_t)kStaticBlocks * 3 * kStaticMaxBins];

// Device address of g_bin_scratch per device, refreshed by every call made
// outside a stream capture with that device current.
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

struct Thresholds {
  long long t[kStaticMaxBins + 1];
};

__device__ __forceinline__ int bin_search(const long long* T, int nk, long long n2) {
  if (n2 < T[0] || n2 >= T[nk]) return -1;
  int lo = 0, hi = nk;   // T[lo] <= n2 < T[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (T[mid] <= n2) lo = mid; else hi = mid;
  }
  return lo;
}

// One warp per row (z, y) of the [N][N][N/2+1] spectrum; n^2 grows along kx,
// so the bins of a 32-lane chunk are contiguous segments: segmented shuffle
// scan, one add per segment into the warp's shared accumulator, fixed-order
// warp and block sums.  Weight 1 on kx = 0 and kx = N/2, 2 elsewhere.
template <typename T>
__global__ void __launch_bounds__(kStaticWarps * 32)
k_bin_rfft(const cx<T>* __restrict__ spec, int n, int nk, double kf, Thresholds thr,
           double* __restrict__ partials) {
  __shared__ double acc_all[kStaticWarps][3 * kStaticMaxBins];
  __shared__ long long T_s[kStaticMaxBins + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = acc_all[warp];
  for (int i = threadIdx.x; i < kStaticWarps * 3 * kStaticMaxBins; i += blockDim.x)
    (&acc_all[0][0])[i] = 0.0;
  for (int i = threadIdx.x; i <= nk; i += blockDim.x) T_s[i] = thr.t[i];
  __syncthreads();
  const unsigned full = 0xffffffffu;
  const int mx = n / 2 + 1;
  const int rows = n * n;
  for (int row = blockIdx.x * kStaticWarps + warp; row < rows; row += gridDim.x * kStaticWarps) {
    const int iz = row / n, iy = row - (row / n) * n;
    const int kz = iz < n / 2 ? iz : iz - n, ky = iy < n / 2 ? iy : iy - n;
    const long long base2 = (long long)kz * kz + (long long)ky * ky;
    const cx<T>* r = spec + (int64_t)row * mx;
    for (int x0 = 0; x0 < mx; x0 += 32) {
      const int kx = x0 + lane;
      double p = 0.0, kk = 0.0, w = 0.0;
      int b = -1;
      if (kx < mx) {
        const cx<T> f = r[kx];
        const long long n2 = base2 + (long long)kx * kx;
        b = bin_search(T_s, nk, n2);
        if (b >= 0) {
          w = (kx == 0 || kx == n / 2) ? 1.0 : 2.0;
          p = w * ((double)f.x * f.x + (double)f.y * f.y);
          kk = w * kf * sqrt((double)n2);
        }
      }
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const double p2 = __shfl_up_sync(full, p, off);
        const double k2 = __shfl_up_sync(full, kk, off);
        const double w2 = __shfl_up_sync(full, w, off);
        const int b2 = __shfl_up_sync(full, b, off);
        if (lane >= off && b2 == b) {
          p += p2;
          kk += k2;
          w += w2;
        }
      }
      const int bn = __shfl_down_sync(full, b, 1);
      if (b >= 0 && (lane == 31 || bn != b)) {
        acc[b] += w;
        acc[nk + b] += kk;
        acc[2 * nk + b] += p;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nk; i += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int wi = 0; wi < kStaticWarps; ++wi) s += acc_all[wi][i];
    partials[(int64_t)blockIdx.x * 3 * nk + i] = s;
  }
}

// out = [count | ksum | psum]; copies the three rows to the caller's buffers.
__global__ void k_bin_static_finish(const double* __restrict__ partials, int nblk, int nk,
                                    double* count, double* ksum, double* psum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nk) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * 3 * nk + i];
  const int row = i / nk, bin = i - row * nk;
  double* dst = row == 0 ? count : (row == 1 ? ksum : psum);
  if (dst) dst[bin] = s;
}

}  // namespace
}  // namespace nupm

using namespace nupm;

extern "C" int pm_bin_power_static(const void* spec, int32_t ngrid, double box, int32_t n_kbins,
                                   int32_t precision, double* count, double* ksum, double* psum,
                                   void* cuda_stream) {
  if (!spec) return PM_ERR_INVALID;
  if (!(ngrid >= 16 && ngrid <= 1024 && (ngrid & (ngrid - 1)) == 0)) return PM_ERR_UNSUPPORTED;
  if (n_kbins < 1 || n_kbins > kStaticMaxBins) {
    fprintf(stderr, "pm_bin_power_static: n_kbins %d exceeds the static maximum %d\n", n_kbins,
            kStaticMaxBins);
    return PM_ERR_RANGE;
  }
  if (!(isfinite(box) && box > 0)) return PM_ERR_INVALID;
  if (precision != PM_FP64 && precision != PM_FP32) return PM_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (s) {   // the scratch address below is the current device's: the stream must be on it
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess || sdev != dev) {
      cudaGetLastError();
      fprintf(stderr, "pm_bin_power_static: the stream is not on the current device\n");
      return PM_ERR_INVALID;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    // host code cannot use the symbol's name as a device address: look it up
    // with the device current, on every call made outside a stream capture
    // (a context created anew after cudaDeviceReset has the array elsewhere);
    // under capture the address of the last uncaptured call is used
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        fprintf(stderr, "pm_bin_power_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return PM_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  Thresholds thr;
  memset(&thr, 0, sizeof thr);
  bin_thresholds(ngrid, n_kbins, thr.t);
  const double kf = 2.0 * M_PI / box;
  if (precision == PM_FP64)
    k_bin_rfft<double><<<kStaticBlocks, kStaticWarps * 32, 0, s>>>(
        static_cast<const cx<double>*>(spec), ngrid, n_kbins, kf, thr, scratch);
  else
    k_bin_rfft<float><<<kStaticBlocks, kStaticWarps * 32, 0, s>>>(
        static_cast<const cx<float>*>(spec), ngrid, n_kbins, kf, thr, scratch);
  k_bin_static_finish<<<(3 * n_kbins + 127) / 128, 128, 0, s>>>(scratch, kStaticBlocks, n_kbins, count,
                                                                  ksum, psum);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}
