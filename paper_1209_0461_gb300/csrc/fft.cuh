// Hand-written 3-D real FFT for the PM grid (sm_103a).
//
// Layout.  The half spectrum of an N^3 real field is kept PACKED: rows of
// M = N/2 complex values, spec[z][y][x2], x2 in [0, M).  Slot x2 = 0 holds
// X[0] + i X[N/2] of the x-transform (both real for real input), so every
// row, column and plane is a power-of-two length.  After the y and z passes
// that slot holds A(ky,kz) + i B(ky,kz), A/B the 2-D spectra of the kx = 0 and
// kx = N/2 planes; consumers unpack them with the Hermitian pair at -k.
//
// One pass = one kernel that streams the whole array once (HBM bound):
//   x pass: rows of N reals <-> M complex (N/2-point complex FFT + split step)
//   y / z pass: W consecutive x2-columns x N elements along a strided axis.
// Inside a CTA each column is transformed by NT = N/E threads that hold E
// elements in registers; radix-R1 x R2 (x R3) Stockham stages exchange data
// through padded shared memory.  Twiddles come from FP64-accurate host tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "consts.cuh"
#include "../../include/nupm.h"

namespace nupm {

constexpr int kFacTableDev = 2048;   // must equal kFacTable (nupm_internal.h)

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.x, -a.y}; }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.x * s, a.y * s}; }

// a * exp(DIR * 2 pi i k / R) with a compile-time R and (after unrolling) k;
// R divides 64 or 192.
template <int R, int DIR, typename T>
__device__ __forceinline__ cx<T> twid_const(cx<T> a, int k) {
  static_assert(64 % R == 0 || 192 % R == 0, "radix must divide 64 or 192");
  if (k == 0) return a;
  if (4 * k == R) return DIR < 0 ? cx<T>{a.y, -a.x} : cx<T>{-a.y, a.x};
  T c, s;
  if constexpr (64 % R == 0) {
    const int j = k * (64 / R);
    c = (T)cos64(j);
    s = (T)DIR * (T)cos64(j + 48);   // sin(t) = cos(t + 3 pi / 2)
  } else {
    const int j = k * (192 / R);
    c = (T)cos192(j);
    s = (T)DIR * (T)cos192(j + 144);
  }
  return {a.x * c - a.y * s, a.x * s + a.y * c};
}

// In-register DFT of length R (2^k or 3 * 2^k, dividing 64 or 192), recursive
// radix-2 decimation in time down to a radix-3 or radix-2 butterfly.
// DIR = -1 forward (exp(-i...)), +1 inverse; unscaled.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 3) {
    // w = exp(DIR 2 pi i / 3): X0 = a + b + c, X1 = a + b w + c w^2,
    // X2 = a + b w^2 + c w^4 = a - (b + c)/2 -/+ DIR i (sqrt 3 / 2)(b - c)
    const cx<T> a = v[0], b = v[1], c = v[2];
    const cx<T> s = b + c, d = b - c;
    const T h = (T)0.86602540378443864676;          // sqrt(3) / 2
    const cx<T> m = {a.x - (T)0.5 * s.x, a.y - (T)0.5 * s.y};
    const cx<T> r = {(T)(-DIR) * h * d.y, (T)DIR * h * d.x};   // DIR i h d
    v[0] = a + s;
    v[1] = m + r;
    v[2] = m - r;
  } else if constexpr (R == 2) {
    const cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else {
    cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<R / 2, DIR>(e);
    dft<R / 2, DIR>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const cx<T> t = twid_const<R, DIR>(o[k], k);
      v[k] = e[k] + t;
      v[k + R / 2] = e[k] - t;
    }
  }
}

// Twiddle W_N^m (forward table exp(-2 pi i m / N)); conjugated for DIR = +1.
__device__ __forceinline__ cx<float> ldg_cx(const cx<float>* p) {
  const float2 q = __ldg(reinterpret_cast<const float2*>(p));
  return {q.x, q.y};
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
  const double2 q = __ldg(reinterpret_cast<const double2*>(p));
  return {q.x, q.y};
}

template <int DIR, typename T>
__device__ __forceinline__ cx<T> twid_table(const cx<T>* __restrict__ tw, int m) {
  cx<T> w = ldg_cx(tw + m);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// Radix plan per (precision, length).  E = R1 elements per thread; R2, R3
// divide R1; NT = L / R1 threads per transform.
template <typename T, int L>
struct Plan;
#define NUPM_PLAN(TT, L_, A, B, C) \
  template <>                      \
  struct Plan<TT, L_> {            \
    static constexpr int R1 = A, R2 = B, R3 = C; \
  };
NUPM_PLAN(float, 8, 8, 1, 1)
NUPM_PLAN(float, 16, 4, 4, 1)
NUPM_PLAN(float, 32, 8, 4, 1)
NUPM_PLAN(float, 64, 8, 8, 1)
NUPM_PLAN(float, 128, 16, 8, 1)
NUPM_PLAN(float, 256, 16, 16, 1)
NUPM_PLAN(float, 512, 32, 16, 1)
NUPM_PLAN(float, 1024, 32, 32, 1)
NUPM_PLAN(float, 96, 12, 4, 2)
NUPM_PLAN(float, 192, 12, 4, 4)
NUPM_PLAN(double, 8, 8, 1, 1)
NUPM_PLAN(double, 16, 4, 4, 1)
NUPM_PLAN(double, 32, 8, 4, 1)
NUPM_PLAN(double, 64, 8, 8, 1)
NUPM_PLAN(double, 128, 16, 8, 1)
NUPM_PLAN(double, 256, 16, 16, 1)
NUPM_PLAN(double, 512, 16, 8, 4)
NUPM_PLAN(double, 1024, 16, 16, 4)
NUPM_PLAN(double, 96, 12, 4, 2)
NUPM_PLAN(double, 192, 12, 4, 4)
#undef NUPM_PLAN

// ---------------------------------------------------------------------------
// Stockham stage on register data.  A transform of length L is split into
// L/R butterflies j; butterfly j (k = j mod NS) reads in[j + i L/R], applies
// W_{NS R}^{i k}, does a radix-R DFT and writes out[(j/NS) NS R + k + i NS].
// Thread t owns butterflies j = t + NT b.  SM provides ld(e)/st(e, v) on the
// thread's own transform in shared memory.
// ---------------------------------------------------------------------------
template <typename T, int L, int E, int NT, int R, int NS, int DIR, bool FIRST, bool LAST, class SM>
__device__ __forceinline__ void stockham_stage(cx<T> (&v)[E], const SM& sm, int t,
                                               const cx<T>* __restrict__ tw) {
  static_assert(E % R == 0, "radix must divide the per-thread element count");
  if constexpr (!FIRST) {
    // gather this stage's inputs (previous stage wrote shared memory)
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + NT * b;
#pragma unroll
      for (int i = 0; i < R; ++i) v[b * R + i] = sm.ld(j + i * (L / R));
    }
    if constexpr (!LAST) __syncthreads();   // reads done before in-place writes
  }
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + NT * b;
    const int k = j % NS;
    if constexpr (NS > 1) {
#pragma unroll
      for (int i = 1; i < R; ++i)
        v[b * R + i] = cmul(v[b * R + i], twid_table<DIR>(tw, i * k * (L / (NS * R))));
    }
    dft<R, DIR>(&v[b * R]);
    if constexpr (!LAST) {
      const int o0 = (j / NS) * NS * R + k;
#pragma unroll
      for (int i = 0; i < R; ++i) sm.st(o0 + i * NS, v[b * R + i]);
    }
  }
  if constexpr (!LAST) __syncthreads();
}

// Full transform of length L held as E = R1 registers per thread.  On entry v
// holds in[t + NT i] (i < E); on exit v[b R_last + i] holds
// out[(t + NT b) + i (L / R_last)].
template <typename T, int L, int DIR, class SM, class P = Plan<T, L>>
__device__ __forceinline__ void fft_regs(cx<T> (&v)[P::R1], const SM& sm, int t,
                                         const cx<T>* __restrict__ tw) {
  constexpr int R1 = P::R1, R2 = P::R2, R3 = P::R3;
  constexpr int E = R1, NT = L / R1;
  if constexpr (R2 == 1) {
    stockham_stage<T, L, E, NT, R1, 1, DIR, true, true>(v, sm, t, tw);
  } else if constexpr (R3 == 1) {
    stockham_stage<T, L, E, NT, R1, 1, DIR, true, false>(v, sm, t, tw);
    stockham_stage<T, L, E, NT, R2, R1, DIR, false, true>(v, sm, t, tw);
  } else {
    stockham_stage<T, L, E, NT, R1, 1, DIR, true, false>(v, sm, t, tw);
    stockham_stage<T, L, E, NT, R2, R1, DIR, false, false>(v, sm, t, tw);
    stockham_stage<T, L, E, NT, R3, R1 * R2, DIR, false, true>(v, sm, t, tw);
  }
}

template <typename T, int L, class P = Plan<T, L>>
__host__ __device__ constexpr int last_radix() {
  return P::R3 > 1 ? P::R3 : (P::R2 > 1 ? P::R2 : P::R1);
}

// Plans with fewer elements per thread for the fused deposit/x kernel: more
// threads per tile for the particle phase and fewer registers, so that the
// shared-memory tile, not the register file, sets the CTAs per SM.
template <typename T, int L>
struct FusedPlan : Plan<T, L> {};
template <>
struct FusedPlan<float, 512> {
  static constexpr int R1 = 16, R2 = 8, R3 = 4;
};
template <>
struct FusedPlan<float, 256> {
  static constexpr int R1 = 8, R2 = 8, R3 = 4;
};

// Shared-memory view of one column of a W-column tile: element e of column c
// at e*W + c + (e >> 5) * PAD (PAD breaks bank conflicts of the stage writes).
template <typename T, int W, int PAD>
struct ColSmem {
  cx<T>* base;
  int c;
  __device__ __forceinline__ cx<T> ld(int e) const { return base[e * W + c + (e >> 5) * PAD]; }
  __device__ __forceinline__ void st(int e, cx<T> v) const { base[e * W + c + (e >> 5) * PAD] = v; }
  static constexpr int words(int L) { return L * W + ((L + 31) >> 5) * PAD; }
};

// Shared-memory view of one row: element e at e + (e >> 5) (one pad per 32).
template <typename T>
struct RowSmem {
  cx<T>* base;
  __device__ __forceinline__ cx<T> ld(int e) const { return base[e + (e >> 5)]; }
  __device__ __forceinline__ void st(int e, cx<T> v) const { base[e + (e >> 5)] = v; }
  static constexpr int words(int L) { return L + ((L + 31) >> 5); }
};

// Column tile width (consecutive x2 columns per CTA) and pad per plan.
template <typename T, int N, int WREQ, class PL = Plan<T, N>>
struct ColCfgW {
  using P = PL;
  static constexpr int M = N / 2;
  static constexpr int E = P::R1;
  static constexpr int NT = N / E;
  // widen small transforms so a CTA has >= 128 threads, never past M columns
  static constexpr int Wt = (WREQ * NT < 128) ? (128 / NT) : WREQ;
  static constexpr int W = Wt > M ? M : Wt;
  static constexpr int THREADS = W * NT;
  static constexpr int PAD = sizeof(T) == 4 ? 8 : 4;
  static constexpr int SMEM_WORDS = ColSmem<T, W, PAD>::words(N);
  // two resident CTAs per SM where the exchange buffer allows it, so one
  // CTA's loads overlap another's math
  static constexpr int MIN_BLOCKS = (size_t)SMEM_WORDS * sizeof(cx<T>) <= 100 * 1024 ? 2 : 1;
};
// Narrow tiles: 64-byte row segments (8 FP32 / 4 FP64 columns); wide tiles:
// 128-byte segments.  Along z a step is an N*M-element stride, and 64-byte
// segments there halve the achieved read bandwidth (measured on GB300), so
// the z passes default to wide tiles from N >= 256 on, the y passes to narrow
// ones; pm_autotune may pick either per pass.
template <typename T, int N>
struct ColNarrow : ColCfgW<T, N, sizeof(T) == 4 ? 8 : 4> {};
template <typename T, int N>
struct ColWide : ColCfgW<T, N, sizeof(T) == 4 ? 16 : 8> {};
template <typename T, int N>
struct ColCfg : ColNarrow<T, N> {};

// Rows per CTA of the x pass.
template <typename T, int N>
struct RowCfg {
  static constexpr int M = N / 2;
  static constexpr int NT = M / Plan<T, M>::R1;
  static constexpr int ROWS = (256 / NT) > 0 ? (256 / NT) : 1;
  static constexpr int THREADS = ROWS * NT;
  static constexpr int ROW_WORDS = RowSmem<T>::words(M);
};

// ---------------------------------------------------------------------------
// y / z pass: transform along a strided axis, in place.
//   data + field * field_stride + blockIdx.y * other_stride + x2 + e * elem_stride
// grid = (M / W, N, nfields)
// ---------------------------------------------------------------------------
// Body of one tile (bx: W-column group, by: the other axis) of field `data`.
template <typename T, int N, int DIR, class Cfg>
__device__ __forceinline__ void fft_col_tile(cx<T>* __restrict__ data, int64_t other_stride, int64_t elem_stride,
                                             const cx<T>* __restrict__ tw, int bx, int by) {
  using P = typename Cfg::P;
  constexpr int E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N, P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  cx<T>* col = data + (int64_t)by * other_stride + (int64_t)bx * W + c;
  ColSmem<T, W, Cfg::PAD> sm{reinterpret_cast<cx<T>*>(smem_raw), c};
  cx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = col[(int64_t)(t + NT * i) * elem_stride];
  fft_regs<T, N, DIR, ColSmem<T, W, Cfg::PAD>, P>(v, sm, t, tw);
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int i = 0; i < RL; ++i)
      col[(int64_t)(t + NT * b + i * (N / RL)) * elem_stride] = v[b * RL + i];
}

// The kernel spells the tile out with the block indices themselves: the same
// code through fft_col_tile's parameters spilled 96 instead of 32-48 bytes a
// thread at 1024-point columns and ran 17% slower on GB300.
template <typename T, int N, int DIR, class Cfg = ColCfg<T, N>>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MIN_BLOCKS)
k_fft_col(cx<T>* __restrict__ data, int64_t other_stride, int64_t elem_stride,
          int64_t field_stride, const cx<T>* __restrict__ tw) {
  using P = typename Cfg::P;
  constexpr int E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N, P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  cx<T>* col = data + (int64_t)blockIdx.z * field_stride + (int64_t)blockIdx.y * other_stride +
               (int64_t)blockIdx.x * W + c;
  ColSmem<T, W, Cfg::PAD> sm{reinterpret_cast<cx<T>*>(smem_raw), c};
  cx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = col[(int64_t)(t + NT * i) * elem_stride];
  fft_regs<T, N, DIR, ColSmem<T, W, Cfg::PAD>, P>(v, sm, t, tw);
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int i = 0; i < RL; ++i)
      col[(int64_t)(t + NT * b + i * (N / RL)) * elem_stride] = v[b * RL + i];
}

// ---------------------------------------------------------------------------
// Inverse z pass with the Green function (a5 + first third of a6).  Columns
// (x2, ky), transform along kz.  Two transforms per tile from the same input
// spectrum (the second read hits L2):
//   out_phi = IFFT_z(G F),   out_dz = IFFT_z(-i D(kz) G F)
// G = gtab[n^2] (x wtab^3 with deconvolution).  The packed column x2 = 0
// (A + i B of the kx = 0 / N/2 planes, whose G differ) comes pre-multiplied
// from plane0[ky][kz] (k_green_plane0).  NOUT = 1: the potential alone (the
// gradient is then taken in real space by the gather).  grid = (M / W, N)
// ---------------------------------------------------------------------------
template <typename T, int N, class Cfg, int NOUT>
__device__ __forceinline__ void fft_z_inv_green_tile(const cx<T>* __restrict__ spec, cx<T>* __restrict__ out_phi,
                                                     cx<T>* __restrict__ out_dz, const cx<T>* __restrict__ plane0,
                                                     const T* __restrict__ gtab, const T* __restrict__ dtab,
                                                     const T* __restrict__ wtab, const cx<T>* __restrict__ tw,
                                                     const float* __restrict__ fac, float fac_inv_du, float coeff,
                                                     int bx, int by) {
  using P = typename Cfg::P;
  constexpr int M = N / 2, E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N, P>();
  constexpr int64_t ES = (int64_t)N * M;   // element stride along z
  constexpr bool kFac = sizeof(T) == 4;    // FP32: G from the fac table, no n^2 gathers
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  float* fac_s = reinterpret_cast<float*>(smem_raw + (size_t)Cfg::SMEM_WORDS * sizeof(cx<T>));
  if constexpr (kFac) {
    for (int j = threadIdx.x; j < kFacTableDev; j += blockDim.x) fac_s[j] = fac[j];
    __syncthreads();
  }
  const int x2 = bx * W + c;
  const int iy = by;
  const int ky = iy < N / 2 ? iy : iy - N;
  const int base2 = ky * ky + x2 * x2;
  const int64_t off = (int64_t)iy * M + x2;
  ColSmem<T, W, Cfg::PAD> sm{reinterpret_cast<cx<T>*>(smem_raw), c};
  const T wyx = wtab ? wtab[iy] * wtab[x2] : (T)1;
  // Green factors of this thread's elements, once per tile, into its own
  // shared-memory slots (layout [i][thread]): keeps them out of registers
  T* gs = reinterpret_cast<T*>(fac_s + (kFac ? kFacTableDev : 0));
  const bool col0 = x2 == 0;
#pragma unroll 1
  for (int i = 0; i < E; ++i) {
    const int iz = t + NT * i;
    const int kz = iz < N / 2 ? iz : iz - N;
    const int n2 = max(base2 + kz * kz, 1);            // >= 1 unless col0
    T g;
    if constexpr (kFac) {
      // G = coeff fac(u) / n^2, u = ln sqrt(n^2), fac linear in u on the table
      const float tt = 0.5f * __logf((float)n2) * fac_inv_du;
      const int j = min((int)tt, kFacTableDev - 2);
      const float fr = tt - (float)j;
      const float fv = fac_s[j] + fr * (fac_s[j + 1] - fac_s[j]);
      g = (T)(coeff * fv / (float)n2);
    } else {
      g = gtab[n2];
    }
    if (wtab) g *= wyx * wtab[iz];
    gs[i * Cfg::THREADS + threadIdx.x] = col0 ? (T)1 : g;
  }
  // branch-free loads: the packed column x2 = 0 reads its pre-multiplied
  // plane0 values (element stride 1), every other column the spectrum
  const cx<T>* src = col0 ? plane0 + (int64_t)iy * N : spec + off;
  const int64_t sstride = col0 ? 1 : ES;
#pragma unroll 1
  for (int pass = 0; pass < NOUT; ++pass) {
    cx<T> v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = src[(int64_t)(t + NT * i) * sstride];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      cx<T> f = cscale(v[i], gs[i * Cfg::THREADS + threadIdx.x]);
      if (pass == 1) {
        const T d = dtab[t + NT * i];
        f = {d * f.y, -d * f.x};                 // -i D(kz) f
      }
      v[i] = f;
    }
    fft_regs<T, N, +1, ColSmem<T, W, Cfg::PAD>, P>(v, sm, t, tw);
    cx<T>* dst = pass == 0 ? out_phi : out_dz;
#pragma unroll
    for (int b = 0; b < E / RL; ++b)
#pragma unroll
      for (int i = 0; i < RL; ++i) dst[off + (int64_t)(t + NT * b + i * (N / RL)) * ES] = v[b * RL + i];
    if (NOUT > 1) __syncthreads();   // the next transform reuses the shared memory
  }
}

template <typename T, int N, class Cfg = ColWide<T, N>, int NOUT = 2>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MIN_BLOCKS)
k_fft_z_inv_green(const cx<T>* __restrict__ spec, cx<T>* __restrict__ out_phi, cx<T>* __restrict__ out_dz,
                  const cx<T>* __restrict__ plane0, const T* __restrict__ gtab, const T* __restrict__ dtab,
                  const T* __restrict__ wtab, const cx<T>* __restrict__ tw, const float* __restrict__ fac,
                  float fac_inv_du, float coeff) {
  fft_z_inv_green_tile<T, N, Cfg, NOUT>(spec, out_phi, out_dz, plane0, gtab, dtab, wtab, tw, fac, fac_inv_du, coeff,
                                        blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Inverse y pass with the y gradient (second third of a6).  Columns (x2, z),
// transform along ky, three transforms per tile:
//   g_dy  = IFFT_y(-i D(ky) g_phi)   (reads g_phi)
//   g_phi = IFFT_y(g_phi)            (re-reads g_phi, L2)
//   g_dz  = IFFT_y(g_dz)
// -i D(ky) is linear, so it acts on the packed column x2 = 0 as on the others.
// grid = (M / W, N)
// ---------------------------------------------------------------------------
template <typename T, int N, class Cfg = ColCfg<T, N>>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MIN_BLOCKS)
k_fft_y_inv_grad(cx<T>* __restrict__ g_phi, cx<T>* __restrict__ g_dy, cx<T>* __restrict__ g_dz,
                 const T* __restrict__ dtab, const cx<T>* __restrict__ tw) {
  using P = typename Cfg::P;
  constexpr int M = N / 2, E = Cfg::E, NT = Cfg::NT, W = Cfg::W, RL = last_radix<T, N, P>();
  constexpr int64_t ES = M;   // element stride along y
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int64_t off = (int64_t)blockIdx.y * N * M + (int64_t)blockIdx.x * W + c;
  ColSmem<T, W, Cfg::PAD> sm{reinterpret_cast<cx<T>*>(smem_raw), c};
#pragma unroll 1
  for (int pass = 0; pass < 3; ++pass) {
    const cx<T>* src = pass == 2 ? g_dz : g_phi;
    cx<T>* dst = pass == 0 ? g_dy : (pass == 1 ? g_phi : g_dz);
    cx<T> v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int iy = t + NT * i;
      cx<T> f = src[off + (int64_t)iy * ES];
      if (pass == 0) {
        const T d = dtab[iy];
        f = {d * f.y, -d * f.x};
      }
      v[i] = f;
    }
    fft_regs<T, N, +1, ColSmem<T, W, Cfg::PAD>, P>(v, sm, t, tw);
#pragma unroll
    for (int b = 0; b < E / RL; ++b)
#pragma unroll
      for (int i = 0; i < RL; ++i) dst[off + (int64_t)(t + NT * b + i * (N / RL)) * ES] = v[b * RL + i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Forward x pass: fixed-point deposit rows -> delta -> packed half spectrum.
//   z[n] = delta[2n] + i delta[2n+1];  Z = FFT_M(z);
//   X[k] = (Z[k] + conj Z[M-k]) / 2 - (i/2) W_N^k (Z[k] - conj Z[M-k]),
//   packed slot 0 = X[0] + i X[M] = (Re Z0 + Im Z0) + i (Re Z0 - Im Z0).
// delta = F * scale - 1 in FP64, rounded to T.  tw_m: W_M^m (m < M);
// tw_n: W_N^k (k < M).  grid = (N^2 / ROWS)
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(RowCfg<T, N>::THREADS)
k_fft_x_fwd(const unsigned long long* __restrict__ grid, cx<T>* __restrict__ spec, double scale,
            const cx<T>* __restrict__ tw_m, const cx<T>* __restrict__ tw_n) {
  using Cfg = RowCfg<T, N>;
  constexpr int M = N / 2, E = Plan<T, M>::R1, NT = M / E, RL = last_radix<T, M>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x % NT;
  const int r = threadIdx.x / NT;
  const int64_t row = (int64_t)blockIdx.x * Cfg::ROWS + r;
  RowSmem<T> sm{reinterpret_cast<cx<T>*>(smem_raw) + r * Cfg::ROW_WORDS};
  const ulonglong2* src = reinterpret_cast<const ulonglong2*>(grid + row * N);
  cx<T> v[E];
  if constexpr (sizeof(T) == 4) {
    // FP32 path: F = hi 2^32 + lo, delta = hi (s 2^32) + (lo s - 1) in FP32 FMAs
    // (absolute error ~ 1e-7; no FP64 arithmetic, which is slow on this part)
    const float hs = (float)(scale * 4294967296.0), ls = (float)scale;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const ulonglong2 q = src[t + NT * i];
      const float ax = fmaf((float)(unsigned)(q.x >> 32), hs, fmaf((float)(unsigned)q.x, ls, -1.0f));
      const float ay = fmaf((float)(unsigned)(q.y >> 32), hs, fmaf((float)(unsigned)q.y, ls, -1.0f));
      v[i] = {(T)ax, (T)ay};
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const ulonglong2 q = src[t + NT * i];
      v[i] = {(T)((double)q.x * scale - 1.0), (T)((double)q.y * scale - 1.0)};
    }
  }
  fft_regs<T, M, -1>(v, sm, t, tw_m);
  // natural-order Z to shared memory for the split step
  if constexpr (Plan<T, M>::R2 > 1) __syncthreads();   // previous stage's readers are done
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int i = 0; i < RL; ++i) sm.st(t + NT * b + i * (M / RL), v[b * RL + i]);
  __syncthreads();
  cx<T>* dst = spec + row * M;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k = t + NT * i;
    const cx<T> zk = sm.ld(k);
    cx<T> out;
    if (k == 0) {
      out = {zk.x + zk.y, zk.x - zk.y};
    } else {
      const cx<T> zm = cconj(sm.ld(M - k));
      const cx<T> ev = cscale(zk + zm, (T)0.5);
      const cx<T> od = cscale(zk - zm, (T)0.5);           // = i O[k]
      const cx<T> w = twid_table<-1>(tw_n, k);
      const cx<T> wo = cmul(w, od);
      out = {ev.x + wo.y, ev.y - wo.x};                     // ev - i * wo
    }
    dst[k] = out;
  }
}

// ---------------------------------------------------------------------------
// Fused a1 + forward x pass.  A CTA owns TZ x TY grid rows (z, y): it
// deposits every particle record of the (TZ+1) x (TY+1) source rows that
// touch them (sorted into rows by k_row_scatter) into a shared-memory tile of
// exact 64-bit sums, then transforms those rows exactly as k_fft_x_fwd.  No
// global deposit grid, no memset, no atomics to DRAM.  With `keep` set the
// tile is also written out (inspection).  grid = (N / TY, N / TZ).
// ---------------------------------------------------------------------------
template <typename T, int N>
struct FusedCfg {
  static constexpr int TZ = 2, TY = 4;
  static constexpr int ROWS = TZ * TY;
  static constexpr int M = N / 2;
  using P = FusedPlan<T, M>;
  static constexpr int E = P::R1;
  static constexpr int NT = M / E;
  static constexpr int THREADS = ROWS * NT;
  static constexpr size_t ACC_BYTES = (size_t)ROWS * N * 8;
  static constexpr size_t XCH_BYTES = (size_t)ROWS * RowSmem<T>::words(M) * sizeof(cx<T>);
  static constexpr size_t SMEM = (ACC_BYTES > XCH_BYTES ? ACC_BYTES : XCH_BYTES);
  // CTAs per SM that the shared-memory tile allows (227 KB), at most 4 (FP32)
  // or 2 (FP64, whose transform needs twice the registers)
  static constexpr int BY_SMEM = (int)((227u * 1024u) / (SMEM + 1024u));
  static constexpr int CAP = sizeof(T) == 4 ? 4 : 2;
  static constexpr int MIN_BLOCKS = BY_SMEM < 1 ? 1 : (BY_SMEM > CAP ? CAP : BY_SMEM);
};

// Exact 64-bit sums on shared memory from native 32-bit atomics: the low
// word's returned old value gives the carry into the high word.  Integer
// addition stays associative, so the sum is bit-exact in any order, and the
// high-word adds may trail the low-word adds of other corners.
__device__ __forceinline__ unsigned int carry_of(unsigned int old, unsigned int lo) {
  return (old + lo < old) ? 1u : 0u;
}

template <typename T, int N>
__device__ __forceinline__ void deposit_fft_x_tile(const unsigned long long* __restrict__ rec,
                                                   const int* __restrict__ row_start, cx<T>* __restrict__ spec,
                                                   double scale, const cx<T>* __restrict__ tw_m,
                                                   const cx<T>* __restrict__ tw_n, unsigned long long* __restrict__ keep,
                                                   int bx, int by, int* status) {
  using Cfg = FusedCfg<T, N>;
  using P = typename Cfg::P;
  constexpr int TZ = Cfg::TZ, TY = Cfg::TY, ROWS = Cfg::ROWS, M = N / 2, E = Cfg::E, NT = Cfg::NT;
  constexpr int RL = last_radix<T, M, P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw);   // 2 x [ROWS][N] words
  // The source rows (tz0-1 .. tz0+TZ-1) x (ty0-1 .. ty0+TY-1) are, per z, one
  // contiguous run of the row-sorted permutation, plus the wrapped row y = N-1
  // when ty0 = 0: NSEG segments, concatenated in a virtual index j.
  constexpr int NSEG = 2 * (TZ + 1);
  __shared__ int seg_pre[NSEG + 1], seg_beg[NSEG];
  const int ty0 = bx * TY, tz0 = by * TZ;
  for (int i = threadIdx.x; i < ROWS * N / 2; i += blockDim.x)
    reinterpret_cast<ulonglong2*>(acc)[i] = ulonglong2{0ull, 0ull};
  // lanes of the (first) warp: all 32, or the whole block when it is smaller
  static_assert(Cfg::THREADS < 32 || Cfg::THREADS % 32 == 0, "whole warps or a single partial warp");
  const unsigned wm = Cfg::THREADS >= 32 ? 0xffffffffu : ((1u << Cfg::THREADS) - 1u);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int len = 0, b0 = 0;
    if (lane < NSEG) {
      const int sz = (tz0 - 1 + lane / 2 + N) % N;
      int r0, r1;
      if (lane & 1) {            // main run of rows
        r0 = sz * N + (ty0 ? ty0 - 1 : 0);
        r1 = sz * N + ty0 + TY;
      } else {                   // wrapped row N-1 (empty unless ty0 = 0)
        r0 = sz * N + N - 1;
        r1 = ty0 ? r0 : r0 + 1;
      }
      b0 = row_start[r0];
      len = row_start[r1] - b0;
    }
    int incl = len;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
      const int o = __shfl_up_sync(wm, incl, d);
      if (lane >= d) incl += o;
    }
    if (lane < NSEG) {
      seg_beg[lane] = b0;
      seg_pre[lane + 1] = incl;
    }
    if (lane == 0) seg_pre[0] = 0;
  }
  __syncthreads();
  const int total = seg_pre[NSEG];
  int bound[NSEG], off[NSEG];   // j >= bound[s] -> record index j + off[s]
#pragma unroll
  for (int k = 0; k < NSEG; ++k) {
    bound[k] = seg_pre[k];
    off[k] = seg_beg[k] - seg_pre[k];
  }
  // low words of the cell sums in one plane, high words in the next: the
  // low-word adds of random x cells spread over all 32 banks
  unsigned int* accw = reinterpret_cast<unsigned int*>(acc);
  constexpr int PLANE = ROWS * N;
  // window rows: z planes tz0-1 .. tz0+TZ-1 (segment / 2), y rows ws .. ws+TY
  // (identified by the record's y cell mod 32; N >= 32 or the mask below)
  static_assert(N < 32 || N % 32 == 0, "the y window is identified mod 32");
  constexpr int YM = (N < 32 ? N : 32) - 1;
  const int ws = (ty0 - 1 + N) % N;
  // A cell's sum wraps past 2^64 only with 65536 or more contributions of up
  // to 2^48 each; a tile with fewer records cannot overflow, and only a tile
  // with more reads back its high-word adds to detect a wrap (PM_ERR_OVERFLOW).
  const bool careful = total >= 65536;
  bool ovf = false;
  constexpr int U = 4;
  for (int j0 = threadIdx.x; j0 < total; j0 += blockDim.x * U) {
    unsigned long long rr[U];
    int zp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * blockDim.x;
      int o = off[0], z = 0;
#pragma unroll
      for (int k = 1; k < NSEG; ++k)
        if (j >= bound[k]) {
          o = off[k];
          z = k >> 1;
        }
      zp[u] = z;
      rr[u] = j < total ? rec[j + o] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j0 + u * (int)blockDim.x >= total) continue;
      const unsigned long long r = rr[u];
      const unsigned wx = (unsigned)r & 0xffffu, wy = (unsigned)(r >> 16) & 0xffffu;
      const unsigned wzz = (unsigned)(r >> 32) & 0xffffu;
      const int cx = (int)(r >> 48) & 0x7ff;
      const int yo = ((int)(r >> 59) - ws) & YM;      // 0 .. TY: row of the window
      const int x1 = cx + 1 == N ? 0 : cx + 1;
      // the particle's (up to) 8 corners in this tile: all low-word adds in
      // flight before any carry is needed
      int slot[8];
      unsigned int lo[8], hi[8], old[8];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const int zl = zp[u] - 1 + dz;
        const unsigned long long wz = dz ? (unsigned long long)wzz : (unsigned long long)(65536u - wzz);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int yl = yo - 1 + dy;
          const bool in = zl >= 0 && zl < TZ && yl >= 0 && yl < TY;
          const unsigned long long wzy = wz * (dy ? (unsigned long long)wy : (unsigned long long)(65536u - wy));
          const int rb = (zl * TY + yl) * N;
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int k = dz * 4 + dy * 2 + dx;
            const unsigned long long v = in ? wzy * (unsigned long long)(dx ? wx : 65536u - wx) : 0ull;
            slot[k] = rb + (dx ? x1 : cx);
            lo[k] = (unsigned int)v;
            hi[k] = (unsigned int)(v >> 32);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (lo[k] | hi[k]) old[k] = atomicAdd(accw + slot[k], lo[k]);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (lo[k] | hi[k]) {
          const unsigned int h = hi[k] + carry_of(old[k], lo[k]);
          if (h) {
            if (careful) {
              const unsigned int oh = atomicAdd(accw + PLANE + slot[k], h);
              ovf = ovf || (oh + h < oh);
            } else {
              atomicAdd(accw + PLANE + slot[k], h);
            }
          }
        }
    }
  }
  if (__syncthreads_or(ovf) && threadIdx.x == 0 && status) atomicCAS(status, 0, PM_ERR_OVERFLOW);
  // forward x transform of the tile's rows (as k_fft_x_fwd)
  const int t = threadIdx.x % NT;
  const int r = threadIdx.x / NT;
  const int gz = tz0 + r / TY, gy = ty0 + r % TY;
  const int64_t grow = (int64_t)gz * N + gy;
  const uint2* lo2 = reinterpret_cast<const uint2*>(accw + r * N);           // cells 2e, 2e+1
  const uint2* hi2 = reinterpret_cast<const uint2*>(accw + PLANE + r * N);
  cx<T> v[E];
  if (keep) {
    ulonglong2* kd = reinterpret_cast<ulonglong2*>(keep + grow * N);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const uint2 l = lo2[t + NT * i], h = hi2[t + NT * i];
      kd[t + NT * i] = ulonglong2{(unsigned long long)l.x | ((unsigned long long)h.x << 32),
                                  (unsigned long long)l.y | ((unsigned long long)h.y << 32)};
    }
  }
  if constexpr (sizeof(T) == 4) {
    // F = hi 2^32 + lo: delta = hi (s 2^32) + (lo s - 1) in FP32 FMAs
    const float hs = (float)(scale * 4294967296.0), ls = (float)scale;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const uint2 l = lo2[t + NT * i], h = hi2[t + NT * i];
      const float ax = fmaf((float)h.x, hs, fmaf((float)l.x, ls, -1.0f));
      const float ay = fmaf((float)h.y, hs, fmaf((float)l.y, ls, -1.0f));
      v[i] = {(T)ax, (T)ay};
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const uint2 l = lo2[t + NT * i], h = hi2[t + NT * i];
      const unsigned long long fa = (unsigned long long)l.x | ((unsigned long long)h.x << 32);
      const unsigned long long fb = (unsigned long long)l.y | ((unsigned long long)h.y << 32);
      v[i] = {(T)((double)fa * scale - 1.0), (T)((double)fb * scale - 1.0)};
    }
  }
  __syncthreads();   // the tile is consumed; its memory now serves the exchange buffers
  RowSmem<T> sm{reinterpret_cast<cx<T>*>(smem_raw) + r * RowSmem<T>::words(M)};
  fft_regs<T, M, -1, RowSmem<T>, P>(v, sm, t, tw_m);
  if constexpr (P::R2 > 1) __syncthreads();
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int i = 0; i < RL; ++i) sm.st(t + NT * b + i * (M / RL), v[b * RL + i]);
  __syncthreads();
  cx<T>* dst = spec + grow * M;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k = t + NT * i;
    const cx<T> zk = sm.ld(k);
    cx<T> out;
    if (k == 0) {
      out = {zk.x + zk.y, zk.x - zk.y};
    } else {
      const cx<T> zm = cconj(sm.ld(M - k));
      const cx<T> ev = cscale(zk + zm, (T)0.5);
      const cx<T> od = cscale(zk - zm, (T)0.5);
      const cx<T> wv = twid_table<-1>(tw_n, k);
      const cx<T> wo = cmul(wv, od);
      out = {ev.x + wo.y, ev.y - wo.x};
    }
    dst[k] = out;
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(FusedCfg<T, N>::THREADS, FusedCfg<T, N>::MIN_BLOCKS)
k_deposit_fft_x(const unsigned long long* __restrict__ rec, const int* __restrict__ row_start,
                cx<T>* __restrict__ spec, double scale, const cx<T>* __restrict__ tw_m, const cx<T>* __restrict__ tw_n,
                unsigned long long* __restrict__ keep, int* status) {
  deposit_fft_x_tile<T, N>(rec, row_start, spec, scale, tw_m, tw_n, keep, blockIdx.x, blockIdx.y, status);
}

// ---------------------------------------------------------------------------
// Inverse x pass, in place: packed half-spectrum rows -> N reals (unscaled),
// fields with bit f of grad_mask set are first multiplied by -i D(kx):
//   Z'[k] = (X[k] + conj X[M-k]) + i W_N^{-k} (X[k] - conj X[M-k]),
//   Z'[0] = (X0 + XM) + i (X0 - XM) with X0 = Re P0, XM = Im P0;
//   z = IFFT_M(Z');  x[2n] = Re z[n], x[2n+1] = Im z[n].
// grid = (rows / ROWS, 1, nfields); rows = N^2.
// ---------------------------------------------------------------------------
// Body of one group of rows (bx) of one field (`data` its base); grad: apply -i D(kx) first.
template <typename T, int N>
__device__ __forceinline__ void fft_x_inv_rows(cx<T>* __restrict__ data, const cx<T>* __restrict__ tw_m,
                                               const cx<T>* __restrict__ tw_n, const T* __restrict__ dtab, bool grad,
                                               int bx) {
  using Cfg = RowCfg<T, N>;
  constexpr int M = N / 2, E = Plan<T, M>::R1, NT = M / E, RL = last_radix<T, M>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x % NT;
  const int r = threadIdx.x / NT;
  const int64_t row = (int64_t)bx * Cfg::ROWS + r;
  RowSmem<T> sm{reinterpret_cast<cx<T>*>(smem_raw) + r * Cfg::ROW_WORDS};
  cx<T>* rowp = data + row * M;
  if (grad) {
    // x gradient first: X'[k] = -i D(k) X[k]; D vanishes on kx = 0 and N/2, so the
    // packed slot 0 (X[0] + i X[N/2]) becomes 0
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = t + NT * i;
      const cx<T> x = rowp[k];
      const T d = k == 0 ? (T)0 : dtab[k];
      sm.st(k, cx<T>{d * x.y, -d * x.x});
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) sm.st(t + NT * i, rowp[t + NT * i]);
  }
  __syncthreads();
  cx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k = t + NT * i;
    const cx<T> xk = sm.ld(k);
    if (k == 0) {
      v[i] = {xk.x + xk.y, xk.x - xk.y};
    } else {
      const cx<T> xm = cconj(sm.ld(M - k));
      const cx<T> s = xk + xm;
      const cx<T> d = cmul(twid_table<+1>(tw_n, k), xk - xm);
      v[i] = {s.x - d.y, s.y + d.x};                       // s + i d
    }
  }
  __syncthreads();   // the stages reuse this row's shared memory
  fft_regs<T, M, +1>(v, sm, t, tw_m);
  T* out = reinterpret_cast<T*>(rowp);
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const int n = t + NT * b + i * (M / RL);
      reinterpret_cast<cx<T>*>(out)[n] = v[b * RL + i];    // (x[2n], x[2n+1])
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(RowCfg<T, N>::THREADS)
k_fft_x_inv(cx<T>* __restrict__ data, int64_t field_stride, const cx<T>* __restrict__ tw_m,
            const cx<T>* __restrict__ tw_n, const T* __restrict__ dtab, int grad_mask) {
  fft_x_inv_rows<T, N>(data + (int64_t)blockIdx.z * field_stride, tw_m, tw_n, dtab, (grad_mask >> blockIdx.z) & 1,
                       blockIdx.x);
}

// ---------------------------------------------------------------------------
// Fused inverse x pass + CIC interpolation + kick (a6 last third + a7).
// Work item = (z slab of TZ particle rows, y segment of LY particle rows).  The
// CTA walks y: at step j it inverse-transforms the x rows (z0 .. z0+TZ, y0+j)
// of the three fields (phi gets -i D(kx) first) into a shared slice, then
// interpolates the particles of rows (z0 .. z0+TZ-1, y0+j-1) from slices j-1
// and j (their 2 x 2 corner rows) and kicks them.  Every particle is handled
// by exactly one CTA, without atomics; the force grids never reach HBM.
// Persistent grid; particle rows from the deposit's row sort.
// ---------------------------------------------------------------------------
template <typename T, int N>
struct XiCfg {
  static constexpr int TZ = 4;
  static constexpr int SLAB = TZ + 1;              // field rows per slice and component
  static constexpr int USED = 3 * SLAB;            // 15 rows per step
  static constexpr int ROWS = 16;
  static constexpr int M = N / 2;
  static constexpr int NT = M / Plan<T, M>::R1;
  static constexpr int THREADS = ROWS * NT;
  static constexpr int LY = N >= 64 ? 32 : N / 2;
  static constexpr size_t XCH = (size_t)ROWS * RowSmem<T>::words(M) * sizeof(cx<T>);
  static constexpr size_t SLICE = (size_t)USED * N * sizeof(T);
  static constexpr size_t SMEM = XCH + 2 * SLICE;
};

template <typename T, int N, class Q>
__global__ void __launch_bounds__(XiCfg<T, N>::THREADS, 1)
k_xinv_interp(const cx<T>* __restrict__ g, int64_t field_elems, const cx<T>* __restrict__ tw_m,
              const cx<T>* __restrict__ tw_n, const T* __restrict__ dtab, const void* __restrict__ pos, int64_t np,
              double delta, const int* __restrict__ row_start, const int* __restrict__ perm, T* __restrict__ vel,
              T kick, T* __restrict__ acc_out, int* status) {
  static_assert((N & (N - 1)) == 0, "the sliding-window gather needs a power-of-two grid");
  using Cfg = XiCfg<T, N>;
  constexpr int M = N / 2, E = Plan<T, M>::R1, NT = Cfg::NT, RL = last_radix<T, M>();
  constexpr int TZ = Cfg::TZ, SLAB = Cfg::SLAB, USED = Cfg::USED, LY = Cfg::LY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* slices = reinterpret_cast<T*>(smem_raw + Cfg::XCH);      // [2][USED][N]
  __shared__ int pre[TZ + 1], beg[TZ];
  const int t = threadIdx.x % NT;
  const int r = threadIdx.x / NT;                              // row group (r == USED: idle duplicate)
  const int comp = (r < USED ? r : 0) / SLAB, zz = (r < USED ? r : 0) % SLAB;
  RowSmem<T> sm{reinterpret_cast<cx<T>*>(smem_raw) + r * RowSmem<T>::words(M)};
  const int ysegs = N / LY;
  const int items = (N / TZ) * ysegs;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int z0 = (item / ysegs) * TZ, y0 = (item % ysegs) * LY;
    for (int j = 0; j <= LY; ++j) {
      const int cur = j & 1;
      const int y = (y0 + j) & (N - 1);
      // ---- inverse x transform of row (z0 + zz, y) of field comp into slice cur
      const cx<T>* rowp = g + (int64_t)comp * field_elems + ((int64_t)((z0 + zz) & (N - 1)) * N + y) * M;
      if (comp == 0) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int k = t + NT * i;
          const cx<T> x = rowp[k];
          const T d = k == 0 ? (T)0 : dtab[k];
          sm.st(k, cx<T>{d * x.y, -d * x.x});
        }
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) sm.st(t + NT * i, rowp[t + NT * i]);
      }
      __syncthreads();
      cx<T> v[E];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = t + NT * i;
        const cx<T> xk = sm.ld(k);
        if (k == 0) {
          v[i] = {xk.x + xk.y, xk.x - xk.y};
        } else {
          const cx<T> xm = cconj(sm.ld(M - k));
          const cx<T> sp = xk + xm;
          const cx<T> dd = cmul(twid_table<+1>(tw_n, k), xk - xm);
          v[i] = {sp.x - dd.y, sp.y + dd.x};
        }
      }
      __syncthreads();
      fft_regs<T, M, +1>(v, sm, t, tw_m);
      if (r < USED) {
        cx<T>* out = reinterpret_cast<cx<T>*>(slices + ((size_t)cur * USED + r) * N);
#pragma unroll
        for (int b = 0; b < E / RL; ++b)
#pragma unroll
          for (int i = 0; i < RL; ++i) out[t + NT * b + i * (M / RL)] = v[b * RL + i];
      }
      if (threadIdx.x == 0 && j >= 1) {
        int run = 0;
        const int py = (y0 + j - 1) & (N - 1);
        for (int q = 0; q < TZ; ++q) {
          const int rr = ((z0 + q) & (N - 1)) * N + py;
          beg[q] = row_start[rr];
          pre[q] = run;
          run += row_start[rr + 1] - row_start[rr];
        }
        pre[TZ] = run;
      }
      __syncthreads();
      // ---- particles of rows (z0 .. z0+TZ-1, y - 1): slices cur^1 (dy = 0) and cur (dy = 1)
      if (j >= 1) {
        const T* s0 = slices + (size_t)(cur ^ 1) * USED * N;
        const T* s1 = slices + (size_t)cur * USED * N;
        const int total = pre[TZ];
        for (int jj = threadIdx.x; jj < total; jj += blockDim.x) {
          int q = 0;
          while (pre[q + 1] <= jj) ++q;
          const int64_t p = perm[beg[q] + (jj - pre[q])];
          int c[3], w[3];
          const typename Q::Raw raw = Q::load(pos, np, p);
          if (!Q::get(raw, N, delta, c, w, status)) continue;
          const T inv = (T)1.0 / (T)65536;
          const T fx1 = (T)w[0] * inv, fy1 = (T)w[1] * inv, fz1 = (T)w[2] * inv;
          const T fx0 = (T)1 - fx1, fy0 = (T)1 - fy1, fz0 = (T)1 - fz1;
          const int zl = (c[2] - z0) & (N - 1);             // 0 .. TZ-1
          const int x0 = c[0], x1 = (c[0] + 1) & (N - 1);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const T* a0 = s0 + (size_t)(d * SLAB + zl) * N;  // (z, y)
            const T* a1 = a0 + N;                             // (z + 1, y)
            const T* b0 = s1 + (size_t)(d * SLAB + zl) * N;  // (z, y + 1)
            const T* b1 = b0 + N;                             // (z + 1, y + 1)
            const T v00 = fx0 * a0[x0] + fx1 * a0[x1];
            const T v01 = fx0 * b0[x0] + fx1 * b0[x1];
            const T v10 = fx0 * a1[x0] + fx1 * a1[x1];
            const T v11 = fx0 * b1[x0] + fx1 * b1[x1];
            const T acc = fz0 * (fy0 * v00 + fy1 * v01) + fz1 * (fy0 * v10 + fy1 * v11);
            vel[d * np + p] += acc * kick;
            if (acc_out) acc_out[d * np + p] = acc;
          }
        }
      }
      __syncthreads();   // slice cur^1 is refilled at the next step
    }
  }
}

}  // namespace nupm
