// Counting sort of the particles by grid row (cz, cy): row key r = cz N + cy.
// The fused deposit/x-transform kernel reads, for its tile of rows, exactly
// the particles that touch it, as packed 8-byte records (cells and weights,
// quantised once here).  The order inside a row follows atomic arrival and
// does not affect any result (integer deposit sums, per-particle gathers).
//
//   k_row_count   warp-aggregated histogram of the keys
//   k_scan_*      exclusive scan of the N^2 counts -> row_start
//   k_row_scatter warp-aggregated cursors -> records (and the permutation)
#pragma once
#include <stdint.h>

#include "grid_kernels.cuh"

namespace nupm {

// Row key of particle p (-1 for an invalid particle; recorded by the count).
// Valid exactly when Quant<T>::cells accepts the particle, with the same cells.
template <typename T>
struct RowKey;

// load() fetches the words the key needs (all of a batch's loads go out before
// any key is computed), key() turns them into the row.
template <>
struct RowKey<float> {
  struct Raw {
    int32_t cy, cz, ox, oy, oz;
  };
  __device__ static __forceinline__ Raw load(const void* pos, int64_t np, int64_t p) {
    const int32_t* q = reinterpret_cast<const int32_t*>(pos);
    return Raw{q[np + p], q[2 * np + p], q[3 * np + p], q[4 * np + p], q[5 * np + p]};
  }
  __device__ static __forceinline__ int key(const Raw& r, int n, double) {
    const float ox = __int_as_float(r.ox), oy = __int_as_float(r.oy), oz = __int_as_float(r.oz);
    if (!(ox >= 0.0f && ox < 1.0f && oy >= 0.0f && oy < 1.0f && oz >= 0.0f && oz < 1.0f)) return -1;
    return wrap_index(r.cz, n) * n + wrap_index(r.cy, n);
  }
};

template <>
struct RowKey<double> {
  struct Raw {
    double x, y, z;
  };
  __device__ static __forceinline__ Raw load(const void* pos, int64_t np, int64_t p) {
    const double* x = reinterpret_cast<const double*>(pos);
    return Raw{x[p], x[np + p], x[2 * np + p]};
  }
  __device__ static __forceinline__ int key(const Raw& r, int n, double delta) {
    const double ux = r.x / delta, uy = r.y / delta, uz = r.z / delta;
    if (!(fabs(ux) < 4503599627370496.0 && fabs(uy) < 4503599627370496.0 && fabs(uz) < 4503599627370496.0))
      return -1;
    const int cy = wrap_index((long long)floor(uy), n), cz = wrap_index((long long)floor(uz), n);
    return cz * n + cy;
  }
};

// Sorted particle record, 8 bytes: bits 0-47 the 16-bit CIC weights of x, y
// and z, bits 48-58 the x cell (N <= 2048), bits 59-63 the y cell mod 32.
// The z cell and the rest of the y cell follow from the record's row.
__device__ __forceinline__ unsigned long long pack_record(const int (&c)[3], const int (&w)[3]) {
  return (unsigned long long)(unsigned)w[0] | ((unsigned long long)(unsigned)w[1] << 16) |
         ((unsigned long long)(unsigned)w[2] << 32) | ((unsigned long long)(unsigned)c[0] << 48) |
         ((unsigned long long)(unsigned)(c[1] & 31) << 59);
}

// Each warp takes kSortBatch x 32 consecutive particles per step (all their
// loads in flight first); the match below sees every lane of the warp.
constexpr int kSortBatch = 4;

// One warp's kSortBatch x 32 particles from `base` on (the warp-uniform body
// of k_row_count; also run by the batched form).
template <typename T>
__device__ __forceinline__ void row_count_warp(const void* __restrict__ pos, int64_t np, int n, double delta,
                                               int* __restrict__ count, int* status, int64_t base) {
  constexpr int U = kSortBatch;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  typename RowKey<T>::Raw raw[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = base + u * 32 + lane;
    if (p < np) raw[u] = RowKey<T>::load(pos, np, p);
  }
  int key[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = base + u * 32 + lane;
    key[u] = p < np ? RowKey<T>::key(raw[u], n, delta) : -2;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const unsigned peers = __match_any_sync(full, key[u]);
    const int leader = __ffs(peers) - 1;
    if (key[u] >= 0 && lane == leader) atomicAdd(count + key[u], __popc(peers));
    if (key[u] == -1) set_status(status, PM_ERR_RANGE);   // skipped by every later stage
  }
}

template <typename T>
__global__ void k_row_count(const void* __restrict__ pos, int64_t np, int n, double delta,
                            int* __restrict__ count, int* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kSortBatch;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * kSortBatch; base < np;
       base += stride)
    row_count_warp<T>(pos, np, n, delta, count, status, base);
}

// One warp's kSortBatch x 32 particles from `base` on (body of k_row_scatter).
template <typename T>
__device__ __forceinline__ void row_scatter_warp(const void* __restrict__ pos, int64_t np, int n, double delta,
                                                 int* __restrict__ cursor, int* __restrict__ perm,
                                                 unsigned long long* __restrict__ rec, int64_t base,
                                                 int* __restrict__ inv = nullptr) {
  constexpr int U = kSortBatch;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  typename Quant<T>::Raw raw[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = base + u * 32 + lane;
    if (p < np) raw[u] = Quant<T>::load(pos, np, p);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = base + u * 32 + lane;
    int c[3] = {0, 0, 0}, w[3] = {0, 0, 0};
    int key = -2;
    if (p < np) key = Quant<T>::cells(raw[u], n, delta, c, w) ? c[2] * n + c[1] : -1;
    const unsigned peers = __match_any_sync(full, key);
    const int leader = __ffs(peers) - 1;
    int start = 0;
    if (key >= 0 && lane == leader) start = atomicAdd(cursor + key, __popc(peers));
    start = __shfl_sync(full, start, leader);
    if (key >= 0) {
      const int slot = start + __popc(peers & ((1u << lane) - 1));
      rec[slot] = pack_record(c, w);
      if (perm) perm[slot] = (int)p;
      if (inv) inv[p] = slot;
    } else if (inv && p < np) {
      inv[p] = -1;   // skipped particle (PM_ERR_RANGE): no slot
    }
  }
}

// Place each valid particle at its row's cursor: the packed record (and, when
// perm is given, the particle index) at the same sorted slot; with inv given,
// each particle's slot (-1 for a skipped particle) in particle order.
template <typename T>
__global__ void k_row_scatter(const void* __restrict__ pos, int64_t np, int n, double delta,
                              int* __restrict__ cursor, int* __restrict__ perm,
                              unsigned long long* __restrict__ rec, int* __restrict__ inv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kSortBatch;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * kSortBatch; base < np;
       base += stride)
    row_scatter_warp<T>(pos, np, n, delta, cursor, perm, rec, base, inv);
}

// Exclusive scan of n values in three launches: per-block scans of 2048
// values (block totals out), a single-block scan of the totals, and the add.
constexpr int kScanBlock = 1024;   // threads; 2 values per thread

__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals,
                              int n);
__global__ void k_scan_totals(int* __restrict__ totals, int nb);
__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ totals, int n, int* __restrict__ cursor);

}  // namespace nupm
