// Counting sort of the particles by grid row (cz, cy): row key r = cz N + cy.
// The fused deposit/x-transform kernel reads, for its tile of rows, exactly
// the particles that touch it.  Only the permutation is stored (perm[i] =
// particle index); the order inside a row follows atomic arrival and does
// not affect any result (integer deposit sums, per-particle interpolation).
//
//   k_row_count   warp-aggregated histogram of the keys
//   k_scan_*      exclusive scan of the N^2 counts -> row_start
//   k_row_scatter warp-aggregated cursors -> perm
#pragma once
#include <stdint.h>

#include "grid_kernels.cuh"

namespace nupm {

// Row key of particle p (-1 for an invalid particle; recorded by the deposit).
template <typename T>
struct RowKey;

template <>
struct RowKey<float> {
  __device__ static __forceinline__ int get(const void* pos, int64_t np, int64_t p, int n, double) {
    const int32_t* q = reinterpret_cast<const int32_t*>(pos);
    const int cy = q[np + p] & (n - 1), cz = q[2 * np + p] & (n - 1);
    const float oy = __int_as_float(q[4 * np + p]), oz = __int_as_float(q[5 * np + p]);
    if (!(oy >= 0.0f && oy < 1.0f && oz >= 0.0f && oz < 1.0f)) return -1;
    return cz * n + cy;
  }
};

template <>
struct RowKey<double> {
  __device__ static __forceinline__ int get(const void* pos, int64_t np, int64_t p, int n, double delta) {
    const double* x = reinterpret_cast<const double*>(pos);
    const double uy = x[np + p] / delta, uz = x[2 * np + p] / delta;
    if (!(fabs(uy) < 4503599627370496.0 && fabs(uz) < 4503599627370496.0)) return -1;
    const int cy = wrap_index((long long)floor(uy), n), cz = wrap_index((long long)floor(uz), n);
    return cz * n + cy;
  }
};

template <typename T>
__global__ void k_row_count(const void* __restrict__ pos, int64_t np, int n, double delta,
                            int* __restrict__ count, int* status) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // whole warps iterate together so the match below sees every lane
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < np; base += stride) {
    const int64_t p = base + lane;
    const int key = p < np ? RowKey<T>::get(pos, np, p, n, delta) : -2;
    const unsigned peers = __match_any_sync(full, key);
    const int leader = __ffs(peers) - 1;
    if (key >= 0 && lane == leader) atomicAdd(count + key, __popc(peers));
    if (key == -1) set_status(status, PM_ERR_RANGE);   // skipped by every later stage
  }
}

template <typename T>
__global__ void k_row_scatter(const void* __restrict__ pos, int64_t np, int n, double delta,
                              int* __restrict__ cursor, int* __restrict__ perm) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < np; base += stride) {
    const int64_t p = base + lane;
    const int key = p < np ? RowKey<T>::get(pos, np, p, n, delta) : -2;
    const unsigned peers = __match_any_sync(full, key);
    const int leader = __ffs(peers) - 1;
    int start = 0;
    if (key >= 0 && lane == leader) start = atomicAdd(cursor + key, __popc(peers));
    start = __shfl_sync(full, start, leader);
    if (key >= 0) perm[start + __popc(peers & ((1u << lane) - 1))] = (int)p;
  }
}

// Exclusive scan of n values in three launches: per-block scans of 2048
// values (block totals out), a single-block scan of the totals, and the add.
constexpr int kScanBlock = 1024;   // threads; 2 values per thread

__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals,
                              int n);
__global__ void k_scan_totals(int* __restrict__ totals, int nb);
__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ totals, int n, int* __restrict__ cursor);

}  // namespace nupm
