// Batched kicks of many boxes of one grid size (FP32 form): every pass of the
// kick is ONE persistent kernel over all boxes.  A pass's work is a list of
// (box, item) pairs -- particle chunks, row tiles, column tiles, response
// panels -- numbered box after box; the CTAs of the launch take the next item
// from an atomic counter (one counter per pass, zeroed at the start of the
// kick; no CTA ever waits on another) and run the same device code as the
// single-box kernels, with the box's own pointers and scalars.  A kick is then
// ~20 launches whatever the number of boxes, and a CUDA graph of it holds
// O(passes) nodes.
//
// Passes (default path of a context: sorted deposit fused with the forward x
// transform, real-space 4-point gradient in the gather):
//   row count, row scan (one CTA per box; it also clears the counts for the
//   next kick), row scatter, deposit + x, y, z, bin sums + their fixed-order
//   reduction, response panels, finish, bin list, fac table, Green plane,
//   Green + z inverse, y inverse, x inverse, gather + kick.
#include <type_traits>
#include <cuda_runtime.h>

#include "fft.cuh"
#include "grid_kernels.cuh"
#include "nu_device.cuh"
#include "nupm_internal.h"
#include "sort.cuh"

namespace nupm {
namespace {

using T = float;
using C = cx<float>;

constexpr int kSortSteps = 4;                  // warp batches per row-sort item and warp
constexpr int kSortChunk = 256 * kSortBatch * kSortSteps;   // particles per row-sort item (a CTA of 256)
constexpr int kFinishGroup = 128;               // bins per finish item
constexpr int kFacGroup = 256;                  // fac-table entries per item
constexpr int kPlaneGroup = 256;                // Green-plane entries per item
constexpr int kScanThreads = 1024;

// The persistent loop: take (box, item) pairs from `counter` until the pass's
// total is reached.  first[b] = the pass's first item of box b, first[nbox] =
// the total; an item's box by bisection of first[].
template <class Pass>
__global__ void __launch_bounds__(Pass::THREADS) k_batch(const BoxArgs* __restrict__ boxes,
                                                        const int* __restrict__ first, int nbox,
                                                        int* __restrict__ counter) {
  __shared__ int s_item;
  const int total = first[nbox];
  for (;;) {
    __syncthreads();   // the previous item is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= total) break;
    int lo = 0, hi = nbox;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (first[mid] <= it) lo = mid; else hi = mid;
    }
    Pass::run(boxes[lo], it - first[lo]);
  }
}

// ---- passes ----
struct PCount {
  static constexpr int THREADS = 256;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) {
#pragma unroll 1
    for (int k = 0; k < kSortSteps; ++k) {
      const int64_t base = (int64_t)item * kSortChunk + (k * 256 + (threadIdx.x & ~31)) * kSortBatch;
      if (base < b.g.np) row_count_warp<T>(b.pos, b.g.np, b.g.n, b.g.delta, b.g.row_count, b.g.status, base);
    }
  }
};

// Exclusive scan of the box's N^2 + 1 row counts into row_start and
// row_cursor by one CTA, kScanPer consecutive values a thread per round
// (16-byte loads and stores) with a carried offset; the counts are cleared
// for the next kick.
constexpr int kScanPer = 16;
struct PScan {
  static constexpr int THREADS = kScanThreads;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int len = b.g.n * b.g.n + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int r0 = 0; r0 < len; r0 += kScanPer * kScanThreads) {
      const int i0 = r0 + kScanPer * tid;
      const bool whole = i0 + kScanPer <= len;   // i0 is a multiple of 16: 16-byte aligned
      int v[kScanPer], s = 0;
      if (whole) {
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) {
          const int4 x = reinterpret_cast<const int4*>(b.g.row_count + i0)[q];
          v[4 * q] = x.x;
          v[4 * q + 1] = x.y;
          v[4 * q + 2] = x.z;
          v[4 * q + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) v[k] = i0 + k < len ? b.g.row_count[i0 + k] : 0;
      }
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) s += v[k];
      int incl = s;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
      }
      if (lane == 31) wsum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const int w0 = wsum[lane];
        int wi = w0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, wi, off);
          if (lane >= off) wi += y;
        }
        wsum[lane] = wi - w0;
      }
      __syncthreads();
      int e = carry_s + wsum[warp] + incl - s;
      int ex[kScanPer];
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        ex[k] = e;
        e += v[k];
      }
      if (whole) {
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) {
          const int4 x = make_int4(ex[4 * q], ex[4 * q + 1], ex[4 * q + 2], ex[4 * q + 3]);
          reinterpret_cast<int4*>(b.g.row_start + i0)[q] = x;
          reinterpret_cast<int4*>(b.g.row_cursor + i0)[q] = x;
          reinterpret_cast<int4*>(b.g.row_count + i0)[q] = make_int4(0, 0, 0, 0);
        }
      } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k)
          if (i0 + k < len) {
            b.g.row_start[i0 + k] = ex[k];
            b.g.row_cursor[i0 + k] = ex[k];
            b.g.row_count[i0 + k] = 0;
          }
      }
      __syncthreads();   // every thread has read carry_s
      if (tid == kScanThreads - 1) carry_s = e;
      __syncthreads();
    }
  }
};

struct PScatter {
  static constexpr int THREADS = 256;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) {
#pragma unroll 1
    for (int k = 0; k < kSortSteps; ++k) {
      const int64_t base = (int64_t)item * kSortChunk + (k * 256 + (threadIdx.x & ~31)) * kSortBatch;
      if (base < b.g.np)
        row_scatter_warp<T>(b.pos, b.g.np, b.g.n, b.g.delta, b.g.row_cursor, b.g.perm, b.g.rec, base, nullptr);
    }
  }
};

template <int N>
struct PDeposit {
  using F = FusedCfg<T, N>;
  static constexpr int THREADS = F::THREADS;
  static constexpr size_t SMEM = F::SMEM;
  __device__ static void run(const BoxArgs& b, int item) {
    constexpr int NX = N / F::TY;
    deposit_fft_x_tile<T, N>(b.g.rec, b.g.row_start, reinterpret_cast<C*>(b.g.spec), b.g.scale,
                             reinterpret_cast<const C*>(b.g.tw_m), reinterpret_cast<const C*>(b.g.tw_n), nullptr,
                             item % NX, item / NX, b.g.status);
  }
};

// Column transforms (narrow tiles) of the spectrum (FIELD = false) or of the
// potential field (FIELD = true), along y or z.
template <int N, int DIR, bool ALONG_Z, bool FIELD>
struct PCol {
  using CC = ColNarrow<T, N>;
  static constexpr int THREADS = CC::THREADS;
  static constexpr size_t SMEM = (size_t)CC::SMEM_WORDS * sizeof(C);
  __device__ static void run(const BoxArgs& b, int item) {
    constexpr int M = N / 2, NX = M / CC::W;
    C* data = reinterpret_cast<C*>(FIELD ? b.g.g : b.g.spec);
    const int64_t other = ALONG_Z ? (int64_t)M : (int64_t)N * M;
    const int64_t elem = ALONG_Z ? (int64_t)N * M : (int64_t)M;
    fft_col_tile<T, N, DIR, CC>(data, other, elem, reinterpret_cast<const C*>(b.g.tw_n), item % NX, item / NX);
  }
};

// Bin sums of rows [item per, (item + 1) per) into partials row `item`.
struct PBins {
  static constexpr int THREADS = kBinWarps * 32;
  __device__ static void run(const BoxArgs& b, int item) {
    const int rows = b.g.n * b.g.n;
    const int per = (rows + b.bin_chunks - 1) / b.bin_chunks;
    const int r0 = item * per, r1 = min(rows, r0 + per);
    bin_power_rows<T, false>(reinterpret_cast<const C*>(b.g.spec), b.g.n, b.nu.nk, b.thr, b.inv_lr, b.kf,
                             b.partials, r0, r1, kBinWarps, item);
  }
};

// psum of each bin: the partials rows summed in a fixed order (32 bins an item).
struct PBinReduce {
  static constexpr int THREADS = kReduceWarps * 32;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) {
    bin_reduce_group(b.partials, b.bin_chunks, b.nu.nk, b.psum, item * 32);
  }
};

// On the side stream: two CTAs per SM at most, so that the passes of the main
// stream keep the rest of each SM (a full-occupancy persistent launch would
// hold every slot until the panels are done and starve them).
struct PPanels {
  static constexpr int THREADS = 128;
  static constexpr size_t SMEM = 0;
  static constexpr int CTAS_PER_SM = 2;
  __device__ static void run(const BoxArgs& b, int item) { nu_panels_item(b.nu, item * 4 + (threadIdx.x >> 5)); }
};

struct PFinish {
  static constexpr int THREADS = kFinishGroup;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) { nu_finish_bin(b.nu, item * kFinishGroup + threadIdx.x); }
};

struct PRlist {
  static constexpr int THREADS = 1024;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int) { nu_rlist_block(b.nu.bins, b.nu.R, b.nu.nk, b.nu.rlist); }
};

struct PFac {
  static constexpr int THREADS = kFacGroup;
  __device__ static void run(const BoxArgs& b, int item) {
    fac_table_entries(const_cast<float*>(b.g.fac), b.fac_umax, b.kf, b.nu.f_nu, b.nu.rlist, b.nu.nk,
                      item * kFacGroup + threadIdx.x, kFacTable);
  }
};

struct PPlane0 {
  static constexpr int THREADS = kPlaneGroup;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) {
    const int i0 = item * kPlaneGroup;
    green_plane0_range<T>(reinterpret_cast<const C*>(b.g.spec), reinterpret_cast<C*>(b.g.plane0), b.g.n,
                          reinterpret_cast<const T*>(b.g.gtab), reinterpret_cast<const T*>(b.g.wtab), b.g.fac,
                          b.g.fac_inv_du, b.g.green_coeff, i0 + threadIdx.x, min(i0 + kPlaneGroup, b.g.n * b.g.n),
                          kPlaneGroup);
  }
};

template <int N>
struct PZInv {
  using CC = ColNarrow<T, N>;
  static constexpr int THREADS = CC::THREADS;
  static constexpr size_t SMEM =
      (size_t)CC::SMEM_WORDS * sizeof(C) + kFacTable * sizeof(float) + (size_t)CC::E * CC::THREADS * sizeof(T);
  __device__ static void run(const BoxArgs& b, int item) {
    constexpr int M = N / 2, NX = M / CC::W;
    C* f = reinterpret_cast<C*>(b.g.g);
    fft_z_inv_green_tile<T, N, CC, 1>(reinterpret_cast<const C*>(b.g.spec), f, f, reinterpret_cast<const C*>(b.g.plane0),
                                      reinterpret_cast<const T*>(b.g.gtab), reinterpret_cast<const T*>(b.g.dtab),
                                      reinterpret_cast<const T*>(b.g.wtab), reinterpret_cast<const C*>(b.g.tw_n),
                                      b.g.fac, b.g.fac_inv_du, b.g.green_coeff, item % NX, item / NX);
  }
};

template <int N>
struct PXInv {
  using RC = RowCfg<T, N>;
  static constexpr int THREADS = RC::THREADS;
  static constexpr size_t SMEM = (size_t)RC::ROWS * RC::ROW_WORDS * sizeof(C);
  __device__ static void run(const BoxArgs& b, int item) {
    fft_x_inv_rows<T, N>(reinterpret_cast<C*>(b.g.g), reinterpret_cast<const C*>(b.g.tw_m),
                         reinterpret_cast<const C*>(b.g.tw_n), reinterpret_cast<const T*>(b.g.dtab), false, item);
  }
};

struct PGather {
  static constexpr int THREADS = kGatherTPB;
  static constexpr size_t SMEM = 0;
  __device__ static void run(const BoxArgs& b, int item) {
    interp_fd_chunk<T>(b.pos, b.g.np, b.g.n, b.g.delta, reinterpret_cast<const T*>(b.g.g),
                       reinterpret_cast<T*>(b.vel), b.kick, nullptr, b.g.status, item);
  }
};

// ---- host side ----
// CTAs per SM of a pass: its CTAS_PER_SM where it sets one, else occupancy
template <class P, class = void>
struct CtaCap {
  static constexpr int v = 0;
};
template <class P>
struct CtaCap<P, std::void_t<decltype(P::CTAS_PER_SM)>> {
  static constexpr int v = P::CTAS_PER_SM;
};

int occupancy_grid(const void* kern, int threads, size_t smem, int sms, int items, int cap) {
  int o = 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
  if (cap > 0 && o > cap) o = cap;
  const int g = (o < 1 ? 1 : o) * sms;
  return items < g ? (items < 1 ? 1 : items) : g;
}

template <class Pass>
void launch_pass(const BatchPlan& p, int pass, size_t smem, cudaStream_t s) {
  const int items = p.h_first[(size_t)pass * (p.nbox + 1) + p.nbox];
  if (items <= 0) return;
  const int grid = occupancy_grid((const void*)k_batch<Pass>, Pass::THREADS, smem, p.sm_count, items, CtaCap<Pass>::v);
  k_batch<Pass><<<grid, Pass::THREADS, smem, s>>>(p.d_boxes, p.d_first + (size_t)pass * (p.nbox + 1), p.nbox,
                                                  p.d_counters + pass);
}

template <int N>
void batch_kick_n(const BatchPlan& p, cudaStream_t s, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  // the response panels read the bins' lattice |k| sums and the history only:
  // they run on the side stream beside the deposit and the transforms
  cudaEventRecord(ev_fork, s);
  cudaStreamWaitEvent(side, ev_fork, 0);
  launch_pass<PPanels>(p, kBpPanels, 0, side);
  cudaEventRecord(ev_join, side);
  launch_pass<PCount>(p, kBpCount, 0, s);
  launch_pass<PScan>(p, kBpScan, 0, s);
  launch_pass<PScatter>(p, kBpScatter, 0, s);
  launch_pass<PDeposit<N>>(p, kBpDeposit, PDeposit<N>::SMEM, s);
  launch_pass<PCol<N, -1, false, false>>(p, kBpY, PCol<N, -1, false, false>::SMEM, s);
  launch_pass<PCol<N, -1, true, false>>(p, kBpZ, PCol<N, -1, true, false>::SMEM, s);
  launch_pass<PBins>(p, kBpBins, kBinWarps * (size_t)p.nk * sizeof(double) + (size_t)(p.nk + 1) * sizeof(int), s);
  launch_pass<PBinReduce>(p, kBpBinReduce, 0, s);
  cudaStreamWaitEvent(s, ev_join, 0);
  launch_pass<PFinish>(p, kBpFinish, 0, s);
  launch_pass<PRlist>(p, kBpRlist, 0, s);
  launch_pass<PFac>(p, kBpFac, 2 * (size_t)p.nk * sizeof(double), s);
  launch_pass<PPlane0>(p, kBpPlane0, 0, s);
  launch_pass<PZInv<N>>(p, kBpZInv, PZInv<N>::SMEM, s);
  launch_pass<PCol<N, +1, false, true>>(p, kBpYInv, PCol<N, +1, false, true>::SMEM, s);
  launch_pass<PXInv<N>>(p, kBpXInv, PXInv<N>::SMEM, s);
  launch_pass<PGather>(p, kBpGather, 0, s);
}

}  // namespace

namespace {
int col_width(int n) {
  switch (n) {
    case 16: return ColNarrow<T, 16>::W;
    case 32: return ColNarrow<T, 32>::W;
    case 64: return ColNarrow<T, 64>::W;
    case 128: return ColNarrow<T, 128>::W;
    case 192: return ColNarrow<T, 192>::W;
    case 256: return ColNarrow<T, 256>::W;
    default: return 0;
  }
}
int row_group(int n) {
  switch (n) {
    case 16: return RowCfg<T, 16>::ROWS;
    case 32: return RowCfg<T, 32>::ROWS;
    case 64: return RowCfg<T, 64>::ROWS;
    case 128: return RowCfg<T, 128>::ROWS;
    case 192: return RowCfg<T, 192>::ROWS;
    case 256: return RowCfg<T, 256>::ROWS;
    default: return 0;
  }
}
}  // namespace

bool batch_supported(int n) { return col_width(n) > 0; }

void batch_items(int n, int64_t np, int nk, int ns, int bin_chunks, int* items) {
  const int m = n / 2;
  items[kBpCount] = items[kBpScatter] = (int)((np + kSortChunk - 1) / kSortChunk);
  items[kBpScan] = 1;
  items[kBpDeposit] = (n / FusedCfg<T, 64>::TY) * (n / FusedCfg<T, 64>::TZ);
  items[kBpY] = items[kBpZ] = items[kBpZInv] = items[kBpYInv] = (m / col_width(n)) * n;
  items[kBpBins] = bin_chunks;
  items[kBpBinReduce] = (nk + 31) / 32;
  items[kBpPanels] = (nk * ns * kNuChunks + 3) / 4;
  items[kBpFinish] = (nk + kFinishGroup - 1) / kFinishGroup;
  items[kBpRlist] = 1;
  items[kBpFac] = (kFacTable + kFacGroup - 1) / kFacGroup;
  items[kBpPlane0] = (n * n + kPlaneGroup - 1) / kPlaneGroup;
  items[kBpXInv] = n * n / row_group(n);
  items[kBpGather] = (int)((np + (int64_t)kGatherTPB * kGatherChunk - 1) / ((int64_t)kGatherTPB * kGatherChunk));
}

int batch_kick(const BatchPlan& p, cudaStream_t s, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  switch (p.n) {
    case 16: batch_kick_n<16>(p, s, side, ev_fork, ev_join); break;
    case 32: batch_kick_n<32>(p, s, side, ev_fork, ev_join); break;
    case 64: batch_kick_n<64>(p, s, side, ev_fork, ev_join); break;
    case 128: batch_kick_n<128>(p, s, side, ev_fork, ev_join); break;
    case 192: batch_kick_n<192>(p, s, side, ev_fork, ev_join); break;
    case 256: batch_kick_n<256>(p, s, side, ev_fork, ev_join); break;
    default: return PM_ERR_UNSUPPORTED;
  }
  return PM_OK;
}

}  // namespace nupm
