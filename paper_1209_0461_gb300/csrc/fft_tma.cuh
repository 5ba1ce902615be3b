// TMA-pipelined column passes (y and z) of the 3-D FFT, persistent CTAs.
//
// Each work item is one W x N column tile of a field.  Thread 0 loads tiles
// with cp.async.bulk.tensor (4-D tensor map: x2, y, z, field) into one of
// two shared buffers; completion is tracked by an mbarrier per buffer.  While
// the CTA transforms item k (registers + padded exchange buffer) and stores
// it, the copy of item k+2 is already in flight, so the HBM stream does not
// stop for the arithmetic.  Items that need two transforms of the same input
// (Green z pass, y-gradient pass) read the staged tile twice from shared
// memory instead of re-reading global memory.
//
// Every wait is bounded: on timeout the kernel records PM_ERR_TIMEOUT, waits
// (bounded) for its own outstanding copies and returns.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "fft.cuh"
#include "grid_kernels.cuh"

namespace nupm {

// kColInvZPhi: the Green z pass with the potential as its only output (the
// gradient then comes from the real-space stencil of the gather)
enum ColMode { kColFwdY = 0, kColFwdZ = 1, kColInvZGreen = 2, kColInvYGrad = 3, kColInvZPhi = 4 };

template <typename T>
struct ColTmaArgs {
  cx<T>* spec;            // packed spectrum (forward passes in place; Green pass input)
  cx<T>* g;               // 3 packed fields
  int64_t field_elems;
  const cx<T>* tw;        // W_N^m
  const cx<T>* plane0;    // Green pass: pre-multiplied packed column x2 = 0, [ky][kz]
  const T* dtab;          // 4-point gradient multiplier per index
  const T* wtab;          // deconvolution (or nullptr)
  const T* gtab;          // FP64 Green table
  const float* fac;       // FP32 fac table
  float fac_inv_du, coeff;
  int* status;
  // bin power sums fused into the forward z pass (k_col_tma_z_fwd<N, true>)
  const int* thr;         // bin thresholds T_0..T_nk of n^2
  float inv_lr;
  int nk;                 // <= kZBinsMaxBins
  double* partials;       // [gridDim.x][nk]: one row per CTA
};

template <typename T, int N>
struct ColTmaCfg {
  static constexpr int M = N / 2;
  static constexpr int E = Plan<T, N>::R1;
  static constexpr int NT = N / E;
  static constexpr int W = sizeof(T) == 4 ? 8 : 4;          // 64-byte row segments
  static constexpr int THREADS = W * NT;
  static constexpr int PAD = ColCfg<T, N>::PAD;
  static constexpr int BOX = N < 256 ? N : 256;             // TMA box extent along the transform
  static constexpr int NBOX = N / BOX;
  static constexpr size_t TILE_BYTES = (size_t)N * W * sizeof(cx<T>);
  static constexpr size_t XCH_BYTES = (size_t)ColSmem<T, W, PAD>::words(N) * sizeof(cx<T>);
  static constexpr size_t FAC_BYTES = sizeof(T) == 4 ? 2048 * sizeof(float) : 0;
  static constexpr size_t SMEM = 2 * TILE_BYTES + XCH_BYTES + FAC_BYTES + 64;
  static constexpr int TILES_PER_ROW = M / W;
};

// Work item -> (field, x2 tile, other index, second transform flag).
template <int MODE>
__device__ __forceinline__ void col_item(int item, int tiles, int tpr, int& field, int& xt, int& other) {
  int k = item;
  field = 0;
  if (MODE == kColInvYGrad && k >= tiles) {   // second half: the d/dz field
    k -= tiles;
    field = 2;
  }
  xt = k % tpr;
  other = k / tpr;
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(ColTmaCfg<T, N>::THREADS, 1)
k_col_tma(const __grid_constant__ CUtensorMap map, ColTmaArgs<T> A) {
  using Cfg = ColTmaCfg<T, N>;
  constexpr int M = N / 2, E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N>();
  constexpr bool AXIS_Z = (MODE == kColFwdZ || MODE == kColInvZGreen);
  constexpr int64_t ES = AXIS_Z ? (int64_t)N * M : (int64_t)M;     // element stride
  constexpr int64_t OS = AXIS_Z ? (int64_t)M : (int64_t)N * M;     // stride of the other index
  constexpr int DIR = (MODE == kColFwdY || MODE == kColFwdZ) ? -1 : +1;
  constexpr bool kFac = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<T>* tile[2] = {reinterpret_cast<cx<T>*>(smem_raw),
                    reinterpret_cast<cx<T>*>(smem_raw + Cfg::TILE_BYTES)};
  cx<T>* xch = reinterpret_cast<cx<T>*>(smem_raw + 2 * Cfg::TILE_BYTES);
  float* fac_s = reinterpret_cast<float*>(smem_raw + 2 * Cfg::TILE_BYTES + Cfg::XCH_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * Cfg::TILE_BYTES + Cfg::XCH_BYTES + Cfg::FAC_BYTES);

  const int tiles = Cfg::TILES_PER_ROW * N;
  const int items = MODE == kColInvYGrad ? 2 * tiles : tiles;
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  ColSmem<T, W, Cfg::PAD> sm{xch, c};

  auto issue = [&](int item, int buf) {
    int field, xt, other;
    col_item<MODE>(item, tiles, Cfg::TILES_PER_ROW, field, xt, other);
    const int xcoord = xt * W * (sizeof(T) == 4 ? 1 : 2);
    mbar_expect_tx(&bar[buf], (uint32_t)Cfg::TILE_BYTES);
#pragma unroll
    for (int bx = 0; bx < Cfg::NBOX; ++bx) {
      cx<T>* dst = tile[buf] + (size_t)bx * Cfg::BOX * W;
      if (AXIS_Z) tma_load_4d(dst, &map, &bar[buf], xcoord, other, bx * Cfg::BOX, field);
      else tma_load_4d(dst, &map, &bar[buf], xcoord, bx * Cfg::BOX, other, field);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if constexpr (MODE == kColInvZGreen && kFac)
    for (int j = threadIdx.x; j < 2048; j += blockDim.x) fac_s[j] = A.fac[j];
  __syncthreads();
  const int first = blockIdx.x, step = gridDim.x;
  if (threadIdx.x == 0) {
    if (first < items) issue(first, 0);
    if (first + step < items) issue(first + step, 1);
  }
  int k = 0;
  for (int item = first; item < items; item += step, ++k) {
    const int buf = k & 1;
    const bool ok = mbar_wait_bounded(&bar[buf], (uint32_t)((k >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicCAS(A.status, 0, PM_ERR_TIMEOUT);
        // let this CTA's own copies finish (bounded) before returning
        mbar_wait_bounded(&bar[buf], (uint32_t)((k >> 1) & 1));
        if (item + step < items) mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
      }
      return;
    }
    int field, xt, other;
    col_item<MODE>(item, tiles, Cfg::TILES_PER_ROW, field, xt, other);
    const int x2 = xt * W + c;
    const cx<T>* st = tile[buf];
    const int ntr = (MODE == kColInvZGreen || (MODE == kColInvYGrad && field == 0)) ? 2 : 1;
    for (int tr = 0; tr < ntr; ++tr) {
      cx<T> v[E];
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = st[(t + NT * i) * W + c];
      if constexpr (MODE == kColInvZGreen) {
        // G delta (tr = 0) and -i D(kz) G delta (tr = 1); packed column x2 = 0
        // takes its pre-multiplied plane0 values instead
        const int iy = other;
        const int ky = iy < N / 2 ? iy : iy - N;
        const int base2 = ky * ky + x2 * x2;
        const T wyx = A.wtab ? A.wtab[iy] * A.wtab[x2] : (T)1;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int iz = t + NT * i;
          cx<T> f;
          if (x2 == 0) {
            f = A.plane0[(int64_t)iy * N + iz];
          } else {
            const int kz = iz < N / 2 ? iz : iz - N;
            const int n2 = base2 + kz * kz;
            T gval;
            if constexpr (kFac) {
              const float tt = 0.5f * __logf((float)n2) * A.fac_inv_du;
              const int j = min((int)tt, 2048 - 2);
              const float fr = tt - (float)j;
              gval = (T)(A.coeff * (fac_s[j] + fr * (fac_s[j + 1] - fac_s[j])) / (float)n2);
            } else {
              gval = A.gtab[n2];
            }
            if (A.wtab) gval *= wyx * A.wtab[iz];
            f = cscale(v[i], gval);
          }
          if (tr == 1) {
            const T d = A.dtab[iz];
            f = {d * f.y, -d * f.x};
          }
          v[i] = f;
        }
      }
      if constexpr (MODE == kColInvYGrad) {
        if (field == 0 && tr == 0) {   // -i D(ky) phi
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const T d = A.dtab[t + NT * i];
            v[i] = {d * v[i].y, -d * v[i].x};
          }
        }
      }
      // all reads of the staged tile done (last transform: the buffer may be
      // refilled) and the previous transform's exchange reads finished
      __syncthreads();
      if (tr == ntr - 1 && threadIdx.x == 0 && item + 2 * step < items) issue(item + 2 * step, buf);
      fft_regs<T, N, DIR>(v, sm, t, A.tw);
      // destination
      cx<T>* dst;
      if constexpr (MODE == kColFwdY || MODE == kColFwdZ) {
        dst = A.spec;
      } else if constexpr (MODE == kColInvZGreen) {
        dst = A.g + (tr == 0 ? 0 : 2 * A.field_elems);
      } else {
        dst = A.g + (field == 2 ? 2 * A.field_elems : (tr == 0 ? A.field_elems : 0));
      }
      dst += (int64_t)other * OS + x2;
#pragma unroll
      for (int b = 0; b < E / RL; ++b)
#pragma unroll
        for (int i = 0; i < RL; ++i) dst[(int64_t)(t + NT * b + i * (N / RL)) * ES] = v[b * RL + i];
    }
  }
}

}  // namespace nupm

namespace nupm {

// ---------------------------------------------------------------------------
// z passes with 128-byte row segments (16 FP32 / 8 FP64 columns) staged by
// TMA in a single shared buffer that afterwards serves as the exchange buffer
// of the transform.  One CTA per SM walks the (x2 tile, y) items; as soon as
// the exchange of item k has been read back (its data now in registers), the
// copy of item k + gridDim.x is issued into the buffer, so it travels while
// item k finishes its butterflies and its stores.  The Green pass takes its
// second transform's input from global memory (the tile it just staged is
// still in L2).
// ---------------------------------------------------------------------------
template <typename T, int N>
struct ColTmaZCfg {
  static constexpr int M = N / 2;
  static constexpr int E = Plan<T, N>::R1;
  static constexpr int NT = N / E;
  static constexpr int W = sizeof(T) == 4 ? 16 : 8;          // 128-byte row segments
  static constexpr int THREADS = W * NT;
  static constexpr int PAD = ColCfg<T, N>::PAD;
  static constexpr int BOX = N < 256 ? N : 256;             // TMA box extent along z
  static constexpr int NBOX = N / BOX;
  static constexpr size_t TILE_BYTES = (size_t)N * W * sizeof(cx<T>);
  static constexpr size_t XCH_BYTES = (size_t)ColSmem<T, W, PAD>::words(N) * sizeof(cx<T>);
  static constexpr size_t BUF_BYTES = XCH_BYTES > TILE_BYTES ? XCH_BYTES : TILE_BYTES;
  static constexpr size_t FAC_BYTES = sizeof(T) == 4 ? 2048 * sizeof(float) : 0;
  static constexpr size_t GS_BYTES = (size_t)E * THREADS * sizeof(T);   // Green factors [E][THREADS]
  static constexpr size_t SMEM = BUF_BYTES + FAC_BYTES + GS_BYTES + 64;
  static constexpr int TILES_PER_ROW = M / W;
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
};

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(ColTmaZCfg<T, N>::THREADS, 1)
k_col_tma_z(const __grid_constant__ CUtensorMap map, ColTmaArgs<T> A) {
  static_assert(MODE == kColFwdZ || MODE == kColInvZGreen || MODE == kColInvZPhi, "z passes only");
  constexpr int NTR = MODE == kColInvZGreen ? 2 : 1;   // transforms per Green tile
  using Cfg = ColTmaZCfg<T, N>;
  constexpr int M = N / 2, E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N>();
  constexpr int64_t ES = (int64_t)N * M;      // element stride along z
  constexpr int DIR = MODE == kColFwdZ ? -1 : +1;
  constexpr bool kFac = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  float* fac_s = reinterpret_cast<float*>(smem_raw + Cfg::BUF_BYTES);
  T* gs = reinterpret_cast<T*>(smem_raw + Cfg::BUF_BYTES + Cfg::FAC_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::BUF_BYTES + Cfg::FAC_BYTES + Cfg::GS_BYTES);
  const int items = Cfg::TILES_PER_ROW * N;   // (x2 tile, y)
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  ColSmem<T, W, Cfg::PAD> sm{buf, c};

  auto issue = [&](int item) {
    const int xt = item % Cfg::TILES_PER_ROW, y = item / Cfg::TILES_PER_ROW;
    const int xcoord = xt * W * (sizeof(T) == 4 ? 1 : 2);
    mbar_expect_tx(bar, (uint32_t)Cfg::TILE_BYTES);
#pragma unroll
    for (int bx = 0; bx < Cfg::NBOX; ++bx)
      tma_load_4d(buf + (size_t)bx * Cfg::BOX * W, &map, bar, xcoord, y, bx * Cfg::BOX, 0);
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if constexpr (MODE != kColFwdZ && kFac)
    for (int j = threadIdx.x; j < 2048; j += blockDim.x) fac_s[j] = A.fac[j];
  __syncthreads();
  const int first = blockIdx.x, step = gridDim.x;
  if (threadIdx.x == 0 && first < items) issue(first);
  int k = 0;
  for (int item = first; item < items; item += step, ++k) {
    if constexpr (MODE != kColFwdZ) {
      // Green factors of this tile (each thread its own slots) while its copy
      // is in flight; the packed column x2 = 0 reads its plane0 values later
      const int x2 = (item % Cfg::TILES_PER_ROW) * W + c, y = item / Cfg::TILES_PER_ROW;
      const int ky = y < N / 2 ? y : y - N;
      const int base2 = ky * ky + x2 * x2;
      const T wyx = A.wtab ? A.wtab[y] * A.wtab[x2] : (T)1;
      if (x2 != 0) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int iz = t + NT * i;
          const int kz = iz < N / 2 ? iz : iz - N;
          const int n2 = base2 + kz * kz;
          T gval;
          if constexpr (kFac) {
            const float tt = 0.5f * __logf((float)n2) * A.fac_inv_du;
            const int j = min((int)tt, 2048 - 2);
            const float fr = tt - (float)j;
            gval = (T)(A.coeff * (fac_s[j] + fr * (fac_s[j + 1] - fac_s[j])) / (float)n2);
          } else {
            gval = A.gtab[n2];
          }
          if (A.wtab) gval *= wyx * A.wtab[iz];
          gs[i * Cfg::THREADS + threadIdx.x] = gval;
        }
      }
    }
    const bool ok = mbar_wait_bounded(bar, (uint32_t)(k & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicCAS(A.status, 0, PM_ERR_TIMEOUT);
        mbar_wait_bounded(bar, (uint32_t)(k & 1));   // this CTA's one copy in flight (bounded)
      }
      return;
    }
    const int xt = item % Cfg::TILES_PER_ROW, y = item / Cfg::TILES_PER_ROW;
    const int x2 = xt * W + c;
    cx<T> v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = buf[(t + NT * i) * W + c];   // the staged tile (dense)
    __syncthreads();   // every read of the tile is done before the exchange overwrites it
    if constexpr (MODE == kColFwdZ) {
      fft_regs<T, N, DIR>(v, sm, t, A.tw);
      fence_proxy_async_shared();
      __syncthreads();   // exchange read back: the buffer may take the next tile
      if (threadIdx.x == 0 && item + step < items) issue(item + step);
      cx<T>* dst = A.spec + (int64_t)y * M + x2;
#pragma unroll
      for (int b = 0; b < E / RL; ++b)
#pragma unroll
        for (int i = 0; i < RL; ++i) dst[(int64_t)(t + NT * b + i * (N / RL)) * ES] = v[b * RL + i];
    } else {
#pragma unroll 1
      for (int tr = 0; tr < NTR; ++tr) {
        if (tr == 1) {   // the second transform reads its input again (L2)
#pragma unroll
          for (int i = 0; i < E; ++i) v[i] = A.spec[(int64_t)(t + NT * i) * ES + (int64_t)y * M + x2];
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int iz = t + NT * i;
          cx<T> f;
          if (x2 == 0) {   // packed column: its pre-multiplied kx = 0 / N/2 values
            f = A.plane0[(int64_t)y * N + iz];
          } else {
            f = cscale(v[i], gs[i * Cfg::THREADS + threadIdx.x]);
          }
          if (tr == 1) {
            const T d = A.dtab[iz];
            f = {d * f.y, -d * f.x};   // -i D(kz)
          }
          v[i] = f;
        }
        if (tr == 1) __syncthreads();   // the first transform's exchange reads are done
        fft_regs<T, N, DIR>(v, sm, t, A.tw);
        if (tr == NTR - 1) {
          fence_proxy_async_shared();
          __syncthreads();
          if (threadIdx.x == 0 && item + step < items) issue(item + step);
        }
        cx<T>* dst = A.g + (tr == 0 ? 0 : 2 * A.field_elems) + (int64_t)y * M + x2;
#pragma unroll
        for (int b = 0; b < E / RL; ++b)
#pragma unroll
          for (int i = 0; i < RL; ++i) dst[(int64_t)(t + NT * b + i * (N / RL)) * ES] = v[b * RL + i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 forward z pass with the exchange in a buffer of its own.  The staged
// tile (N x 16 columns, 128-byte row segments, the same tensor map as
// k_col_tma_z) is read into registers and the next tile's copy is issued at
// once, so that it travels during this tile's butterflies and stores
// (k_col_tma_z can issue it only once the exchange, which reuses the tile
// buffer, has been read back).  The exchange buffer holds 8 of the 16
// columns: the two halves exchange in turn.  The same butterflies as fft_regs
// for the two-stage plans of 256, 512 and 1024 points (one exchange).
//
// BINS: the power sums of the spectrum's bins (a3) in the same pass.  A
// tile's |delta_k|^2 go to the exchange buffer (free after the exchange), and
// one warp per column folds them at kz = 0 into rings j = |kz| (n^2 =
// ky^2 + x2^2 + j^2, weight 2 for the +-kx pair) for bin_rings_warp; the
// packed column x2 = 0 is left to k_bin_plane0.  Each CTA keeps one
// float-pair accumulator per warp and writes their sum in FP64, in warp
// order, to its row of partials at the end: a fixed order for a fixed grid.
// ---------------------------------------------------------------------------
constexpr int kZBinsMaxBins = 256;

template <int N, bool BINS>
struct ColTmaZFwdCfg {
  using T = float;
  using P = Plan<T, N>;
  static constexpr int M = N / 2;
  static constexpr int E = P::R1, R2 = P::R2;
  static constexpr int NT = N / E;
  static constexpr int W = ColTmaZCfg<T, N>::W, WH = W / 2;
  static constexpr int THREADS = W * NT;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int PAD = ColTmaZCfg<T, N>::PAD;
  static constexpr int BOX = ColTmaZCfg<T, N>::BOX;
  static constexpr int NBOX = N / BOX;
  static constexpr size_t TILE_BYTES = (size_t)N * W * sizeof(cx<T>);
  static constexpr size_t XCH_BYTES = (size_t)ColSmem<T, WH, PAD>::words(N) * sizeof(cx<T>);
  static constexpr size_t ACC_BYTES = BINS ? (size_t)WARPS * kZBinsMaxBins * sizeof(float2) : 0;
  static constexpr size_t SMEM = TILE_BYTES + XCH_BYTES + ACC_BYTES + 64;
  static constexpr int TILES_PER_ROW = M / W;
  static_assert(P::R3 == 1 && R2 > 1 && E % R2 == 0, "two-stage plans only");
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
  static_assert(TILE_BYTES % 128 == 0 && (TILE_BYTES + XCH_BYTES + ACC_BYTES) % 8 == 0, "buffer alignment");
  static_assert(!BINS || (size_t)W * N * sizeof(float) <= XCH_BYTES, "the powers fit the exchange buffer");
  static_assert(!BINS || (N / 2) % 32 == 0, "rings per lane");
};

template <int N, bool BINS>
__global__ void __launch_bounds__(ColTmaZFwdCfg<N, BINS>::THREADS, 1)
k_col_tma_z_fwd(const __grid_constant__ CUtensorMap map, ColTmaArgs<float> A) {
  using T = float;
  using Cfg = ColTmaZFwdCfg<N, BINS>;
  constexpr int M = N / 2, E = Cfg::E, R2 = Cfg::R2, NT = Cfg::NT, W = Cfg::W, WH = Cfg::WH;
  constexpr int64_t ES = (int64_t)N * M;      // element stride along z
  constexpr int DIR = -1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* xch = reinterpret_cast<cx<T>*>(smem_raw + Cfg::TILE_BYTES);
  float2* acc_all = reinterpret_cast<float2*>(smem_raw + Cfg::TILE_BYTES + Cfg::XCH_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::TILE_BYTES + Cfg::XCH_BYTES + Cfg::ACC_BYTES);
  const int items = Cfg::TILES_PER_ROW * N;   // (x2 tile, y)
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int half = c / WH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ColSmem<T, WH, Cfg::PAD> xs{xch, c % WH};

  auto issue = [&](int item) {
    const int xt = item % Cfg::TILES_PER_ROW, y = item / Cfg::TILES_PER_ROW;
    mbar_expect_tx(bar, (uint32_t)Cfg::TILE_BYTES);
#pragma unroll
    for (int bx = 0; bx < Cfg::NBOX; ++bx)
      tma_load_4d(tile + (size_t)bx * Cfg::BOX * W, &map, bar, xt * W, y, bx * Cfg::BOX, 0);
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if constexpr (BINS)
    for (int i = threadIdx.x; i < Cfg::WARPS * A.nk; i += blockDim.x) acc_all[i] = make_float2(0.0f, 0.0f);
  __syncthreads();
  const int first = blockIdx.x, step = gridDim.x;
  if (threadIdx.x == 0 && first < items) issue(first);
  int k = 0;
  for (int item = first; item < items; item += step, ++k) {
    const bool ok = mbar_wait_bounded(bar, (uint32_t)(k & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicCAS(A.status, 0, PM_ERR_TIMEOUT);
        mbar_wait_bounded(bar, (uint32_t)(k & 1));   // this CTA's one copy in flight (bounded)
      }
      return;
    }
    const int xt = item % Cfg::TILES_PER_ROW, y = item / Cfg::TILES_PER_ROW;
    const int x2 = xt * W + c;
    cx<T> v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = tile[(t + NT * i) * W + c];   // the staged tile (dense)
    fence_proxy_async_shared();
    __syncthreads();   // every read of the tile is done: it may take the next copy
    if (threadIdx.x == 0 && item + step < items) issue(item + step);
    // first stage: radix-E butterfly on the thread's elements t + NT i
    dft<E, DIR>(v);
    // the exchange, one half of the columns at a time
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (half == h) {
#pragma unroll
        for (int i = 0; i < E; ++i) xs.st(t * E + i, v[i]);
      }
      __syncthreads();
      if (half == h) {
#pragma unroll
        for (int b = 0; b < E / R2; ++b) {
          const int j = t + NT * b;
#pragma unroll
          for (int i = 0; i < R2; ++i) v[b * R2 + i] = xs.ld(j + i * (N / R2));
        }
      }
      __syncthreads();
    }
    // second stage: twiddles W_N^{i k}, k = j mod E, and radix-R2 butterflies
#pragma unroll
    for (int b = 0; b < E / R2; ++b) {
      const int j = t + NT * b;
      const int kk = j % E;
#pragma unroll
      for (int i = 1; i < R2; ++i) v[b * R2 + i] = cmul(v[b * R2 + i], twid_table<DIR>(A.tw, i * kk * (N / (E * R2))));
      dft<R2, DIR>(&v[b * R2]);
    }
    cx<T>* dst = A.spec + (int64_t)y * M + x2;
#pragma unroll
    for (int b = 0; b < E / R2; ++b)
#pragma unroll
      for (int i = 0; i < R2; ++i) dst[(int64_t)(t + NT * b + i * (N / R2)) * ES] = v[b * R2 + i];
    if constexpr (BINS) {
      constexpr int J = N / 2, ER = J / 32;
      // |delta_k|^2 of this tile, element iz of column c at iz W + ((c + iz / ER) mod W):
      // the stores of a warp (16 columns, two consecutive iz) and the ring
      // loads of a warp (one column, lanes ER apart in iz) fall in distinct
      // banks, two lanes a bank for the loads
      static_assert(W == 16, "the rotation assumes 16 columns");
      float* pw = reinterpret_cast<float*>(xch);
      auto at = [&](int iz, int col) { return iz * W + ((col + iz / ER) & (W - 1)); };
#pragma unroll
      for (int b = 0; b < E / R2; ++b)
#pragma unroll
        for (int i = 0; i < R2; ++i) {
          const cx<T> q = v[b * R2 + i];
          pw[at(t + NT * b + i * (N / R2), c)] = q.x * q.x + q.y * q.y;
        }
      __syncthreads();
      const int ky = y < N / 2 ? y : y - N;
      for (int col = warp; col < W; col += Cfg::WARPS) {
        const int x2c = xt * W + col;
        if (x2c == 0) continue;                      // the packed column: k_bin_plane0
        float r[ER];
#pragma unroll
        for (int i = 0; i < ER; ++i) {
          const int j = lane * ER + i;                // j < J: kz = j and kz = -j
          r[i] = 2.0f * (j > 0 ? pw[at(j, col)] + pw[at(N - j, col)] : pw[at(0, col)]);
        }
        const int base2 = ky * ky + x2c * x2c;
        bin_rings_warp<ER>(r, base2, true, base2 + J * J, 2.0f * pw[at(J, col)], A.thr, A.nk, A.inv_lr,
                           acc_all + warp * A.nk);
      }
      __syncthreads();   // the powers are read before the next tile's exchange
    }
  }
  if constexpr (BINS) {
    __syncthreads();
    for (int i = threadIdx.x; i < A.nk; i += blockDim.x) {
      double sum = 0.0;
      for (int w = 0; w < Cfg::WARPS; ++w) sum += (double)acc_all[w * A.nk + i].x + (double)acc_all[w * A.nk + i].y;
      A.partials[(int64_t)blockIdx.x * A.nk + i] = sum;
    }
  }
}

}  // namespace nupm
