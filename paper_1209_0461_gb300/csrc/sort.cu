// Exclusive scan of the row counts (row_start) for the particle row sort.
#include <cuda_runtime.h>

#include "sort.cuh"

namespace nupm {

// Block b scans in[b*2048 .. b*2048+2047] (exclusive) into out, total -> totals[b].
__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals, int n) {
  __shared__ int warp_sum[kScanBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 2 * kScanBlock + 2 * tid;
  const int a = i0 < n ? in[i0] : 0;
  const int b = i0 + 1 < n ? in[i0 + 1] : 0;
  int s = a + b;
  int incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_sum[lane];
    int wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    warp_sum[lane] = wi - w;   // exclusive warp offsets
    if (lane == 31) totals[blockIdx.x] = wi;
  }
  __syncthreads();
  const int excl = warp_sum[warp] + incl - s;
  if (i0 < n) out[i0] = excl;
  if (i0 + 1 < n) out[i0 + 1] = excl + a;
}

// Single block: exclusive scan of nb <= 2 * kScanBlock block totals, in place.
__global__ void k_scan_totals(int* __restrict__ totals, int nb) {
  __shared__ int warp_sum[kScanBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int a = 2 * tid < nb ? totals[2 * tid] : 0;
  const int b = 2 * tid + 1 < nb ? totals[2 * tid + 1] : 0;
  const int s = a + b;
  int incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_sum[lane];
    int wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    warp_sum[lane] = wi - w;
  }
  __syncthreads();
  const int excl = warp_sum[warp] + incl - s;
  if (2 * tid < nb) totals[2 * tid] = excl;
  if (2 * tid + 1 < nb) totals[2 * tid + 1] = excl + a;
}

// out[i] += offset of its block; cursor[i] = out[i].
__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ totals, int n, int* __restrict__ cursor) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int v = out[i] + totals[i / (2 * kScanBlock)];
    out[i] = v;
    cursor[i] = v;
  }
}

}  // namespace nupm
