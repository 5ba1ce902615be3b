// Particle and spectrum kernels of the PM kick (sm_103a), templated on the
// grid precision T (float: PM_FP32, double: PM_FP64).
//
//   k_deposit      fixed-point CIC scatter (Sec. 4.3 (ii)), 64-bit integer atomics
//   k_bin_power    per-|k|-bin sums of the forward spectrum (P_cdm, Sec. 4.3 (ii))
//   k_green        delta_M = delta_cdm [(1-f) + f R(|k|)] (Eq. phases, Sec. 4.3 (iv)),
//                  Poisson (Eq. Poisson), 4-point gradient -> 3 spectra
//   k_interp_kick  CIC gather of the 3 force grids, u += acc * K
//   k_unpack_spec  packed half spectrum -> rfftn layout (inspection only)
#pragma once
#include <stdint.h>

#include <type_traits>

#include "async_copy.cuh"
#include "fft.cuh"
#include "nupm_internal.h"

namespace nupm {

constexpr int kWeightBits = 16;
constexpr int kWeightOne = 1 << kWeightBits;

// Record the first device-side error (status 0 -> code).
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Periodic wrap onto [0, n): a mask for powers of two, else the floored
// remainder (32-bit for int cells, 64-bit only for FP64 cell numbers).
__device__ __forceinline__ int wrap_index(int c, int n) {
  if ((n & (n - 1)) == 0) return c & (n - 1);
  const int r = c % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ int wrap_index(long long c, int n) {
  if ((n & (n - 1)) == 0) return (int)(c & (long long)(n - 1));
  const long long r = c % n;
  return (int)(r < 0 ? r + n : r);
}
// (n - i) mod n for i in [0, n): the index of the Hermitian partner.
__device__ __forceinline__ int partner_index(int i, int n) { return i == 0 ? 0 : n - i; }

// Quantised particle: cell (wrapped) and 16-bit weight per axis.  load()
// fetches the raw position words, get() turns them into (cell, weight) and
// returns false (recording PM_ERR_RANGE) for an invalid particle.  Keeping
// the two apart lets a thread put several particles' loads in flight at once.
template <typename T>
struct Quant;

template <>
struct Quant<double> {   // FP64 comoving positions, double[3][np]
  struct Raw {
    double x[3];
  };
  __device__ static __forceinline__ Raw load(const void* pos, int64_t np, int64_t p) {
    const double* x = reinterpret_cast<const double*>(pos);
    return Raw{{x[p], x[np + p], x[2 * np + p]}};
  }
  __device__ static __forceinline__ bool cells(const Raw& r, int n, double delta, int (&c)[3], int (&w)[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double u = r.x[d] / delta;                 // same IEEE division as the definition
      if (!(fabs(u) < 4503599627370496.0)) return false;   // non-finite or |u| >= 2^52
      const double cf = floor(u);
      const double o = u - cf;                         // exact
      w[d] = (int)floor(o * (double)kWeightOne);
      c[d] = wrap_index((long long)cf, n);
    }
    return true;
  }
  __device__ static __forceinline__ bool get(const Raw& r, int n, double delta, int (&c)[3], int (&w)[3],
                                             int* status) {
    if (cells(r, n, delta, c, w)) return true;
    set_status(status, PM_ERR_RANGE);
    return false;
  }
};

template <>
struct Quant<float> {    // int32 words [6][np]: cells rows 0-2, FP32 offsets rows 3-5
  struct Raw {
    int32_t q[6];
  };
  __device__ static __forceinline__ Raw load(const void* pos, int64_t np, int64_t p) {
    const int32_t* q = reinterpret_cast<const int32_t*>(pos);
    Raw r;
#pragma unroll
    for (int d = 0; d < 6; ++d) r.q[d] = q[d * np + p];
    return r;
  }
  __device__ static __forceinline__ bool cells(const Raw& r, int n, double, int (&c)[3], int (&w)[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float o = __int_as_float(r.q[3 + d]);
      if (!(o >= 0.0f && o < 1.0f)) return false;
      w[d] = (int)floorf(o * (float)kWeightOne);       // exact scaling by 2^16
      c[d] = wrap_index((int)r.q[d], n);
    }
    return true;
  }
  __device__ static __forceinline__ bool get(const Raw& r, int n, double delta, int (&c)[3], int (&w)[3],
                                             int* status) {
    if (cells(r, n, delta, c, w)) return true;
    set_status(status, PM_ERR_RANGE);
    return false;
  }
};

constexpr int kDepositBatch = 4;   // particles per thread per iteration
constexpr int kInterpBatch = 2;

// ---------------------------------------------------------------------------
// a1: CIC deposit.  Corner (dx,dy,dz) of cell c gets prod_d (dx ? w_d : 2^16 - w_d).
// Integer addition is associative, so the grid is bit-exact in any order.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_deposit(const void* __restrict__ pos, int64_t np, int n, double delta,
                          unsigned long long* __restrict__ grid, int* status) {
  constexpr int U = kDepositBatch;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < np; p0 += stride * U) {
    typename Quant<T>::Raw raw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * stride;
      if (p < np) raw[u] = Quant<T>::load(pos, np, p);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int c[3], w[3];
      if (p0 + u * stride >= np || !Quant<T>::get(raw[u], n, delta, c, w, status)) continue;
      const unsigned long long wx[2] = {(unsigned long long)(kWeightOne - w[0]), (unsigned long long)w[0]};
      const unsigned long long wy[2] = {(unsigned long long)(kWeightOne - w[1]), (unsigned long long)w[1]};
      const unsigned long long wz[2] = {(unsigned long long)(kWeightOne - w[2]), (unsigned long long)w[2]};
      const int x1 = c[0] + 1 == n ? 0 : c[0] + 1;
      const int y1 = c[1] + 1 == n ? 0 : c[1] + 1;
      const int z1 = c[2] + 1 == n ? 0 : c[2] + 1;
      const int xs[2] = {c[0], x1}, ys[2] = {c[1], y1}, zs[2] = {c[2], z1};
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const unsigned long long wzy = wz[dz] * wy[dy];
          const int64_t rowi = ((int64_t)zs[dz] * n + ys[dy]) * n;
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const unsigned long long wt = wzy * wx[dx];
            if (wt) {
              const unsigned long long o = atomicAdd(grid + rowi + xs[dx], wt);
              if (o + wt < o) set_status(status, PM_ERR_OVERFLOW);   // the cell's sum wrapped past 2^64
            }
          }
        }
    }
  }
}

// Signed frequency of index i on an n-point axis.
__device__ __forceinline__ int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// ---------------------------------------------------------------------------
// a3: binned power of the packed spectrum, deterministic.  One warp per row
// (z, y); lane L takes the E = ceil(M / 32) consecutive x2 from L E.  Along a
// row n^2 = kz^2 + ky^2 + x2^2 grows with x2, so a lane's modes fall into runs
// of equal bin, and the lanes' runs follow each other in bin order:
//   * a run that neither starts nor ends the lane's range holds every mode of
//     its bin in this row: the lane adds it to the warp's accumulator;
//   * the first and the last run of each lane may continue into neighbouring
//     lanes: a segmented shuffle scan over the lanes' last runs (a lane whose
//     range is one run passes the sum through) joins them, and each joined
//     segment is added once, by the lane where it ends (a lane with several
//     runs closes the incoming segment with its first run).
// Every add has one writer in a fixed order, so the sums are reproducible;
// warps and CTAs are then summed in a fixed order (k_bin_reduce).
// The bin of n^2 is the b with T_b <= n^2 < T_{b+1} (integer thresholds in
// shared memory): floor(nk ln n^2 / ln r^2) for the lane's first mode,
// corrected against T, then advanced while n^2 >= T_{b+1}.
//   LATTICE = true : accumulate the mode count sum w and sum w |k| (depends on
//                    the lattice only; run once per context)
//   LATTICE = false: accumulate sum w |delta_k|^2 in the grid precision T
//                    along runs and lanes, one FP64 add per run or segment
// The packed slot x2 = 0 is unpacked with the row at (-z, -y):
//   A = (F(k) + conj F(-k)) / 2   (kx = 0),  B = (F(k) - conj F(-k)) / (2i)  (kx = N/2).
// Shared memory: [kBinWarps][NV][nk] doubles (NV = 2 lattice sums or 1), then
// T[0..nk].
// ---------------------------------------------------------------------------
constexpr int kBinWarps = 4;
constexpr int kBinLaneMax = 16;   // modes per lane (M <= 512)

__device__ __forceinline__ int bin_of_n2(int n2, const int* T, int nk, float inv_lr) {
  int b = (int)(__logf((float)n2) * inv_lr);
  b = min(max(b, 0), nk - 1);
  while (b < nk - 1 && T[b + 1] <= n2) ++b;
  while (b > 0 && T[b] > n2) --b;
  return (T[b] <= n2 && n2 < T[b + 1]) ? b : -1;
}

// FP32 power sums accumulate per bin as an unevaluated pair hi + lo of// FP32 power sums accumulate per bin as an unevaluated pair hi + lo of
// floats (error-free two-sum of each added run or segment): about twice
// float precision without GB300's narrow FP64 pipe, which otherwise limits
// the kernel.  The pair is summed into FP64 once per CTA.
template <typename T, bool LATTICE>
constexpr bool kBinPair = !LATTICE && sizeof(T) == 4;

__device__ __forceinline__ void pair_add(float2* a, float x) {
  float2 v = *a;
  const float s = v.x + x;
  const float bp = s - v.x;
  const float err = (v.x - (s - bp)) + (x - bp);
  v.x = s;
  v.y += err;
  *a = v;
}

// Power sums of one warp over "rings" j of a line of modes whose n^2 =
// base2 + j^2 grows with j (the modes along z of one (x2, y) column, folded
// at kz = 0, or along y of one kz row): lane l holds the values r[i] of rings
// j = l ER + i, and the last lane also `extra` for the ring n2x after all of
// them.  The bins of a lane's rings are monotone and the lanes' ranges follow
// each other, so each lane sums its runs of equal bin in order, a bin met only
// inside one lane is added at once, and the runs that cross lanes are joined
// by one segmented scan (as bin_row_staged); every bin gets its adds in a fixed
// order, into the warp's float-pair accumulator acc[nk] (pair_add).
template <int ER>
__device__ __forceinline__ void bin_rings_warp(const float (&r)[ER], int base2, bool has_extra, int n2x,
                                               float extra, const int* __restrict__ T, int nk, float inv_lr,
                                               float2* acc) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int j0 = lane * ER;
  const int n20 = base2 + j0 * j0;
  int bL = bin_of_n2(n20 > 0 ? n20 : 1, T, nk, inv_lr);   // n^2 = 0 (the mean) carries no power
  const int bF = bL;
  int tnext = T[bL + 1];
  bool multi = false;
  float sF = 0.0f, c = 0.0f;
  auto ring = [&](int n2m, float v) {
    if (n2m >= tnext) {
      if (!multi) {          // the first run waits for the lane combine
        sF = c;
        multi = true;
      } else {               // an inner run: a bin no other lane has
        pair_add(acc + bL, c);
      }
      c = 0.0f;
      do {
        ++bL;
        tnext = T[bL + 1];
      } while (n2m >= tnext);
    }
    c += v;
  };
#pragma unroll
  for (int i = 0; i < ER; ++i) {
    const int j = j0 + i;
    ring(base2 + j * j, r[i]);
  }
  if (lane == 31 && has_extra) ring(n2x, extra);
  int kk = (bL << 1) | (multi ? 0 : 1);   // key, open (a single-run lane continues the previous one)
  float s0 = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int pkk = __shfl_up_sync(full, kk, off);
    const float p0 = __shfl_up_sync(full, s0, off);
    if (lane >= off && (kk & 1) && (pkk >> 1) == (kk >> 1)) {
      s0 += p0;
      kk = (kk & ~1) | (pkk & 1);
    }
  }
  const int k = kk >> 1;
  const int qk = __shfl_up_sync(full, k, 1);
  const float q0 = __shfl_up_sync(full, s0, 1);
  const int nextF = __shfl_down_sync(full, bF, 1);
  __syncwarp();
  if (multi) pair_add(acc + bF, sF + ((lane > 0 && qk == bF) ? q0 : 0.0f));
  __syncwarp();
  if (lane == 31 || nextF != k) pair_add(acc + k, s0);
  __syncwarp();
}

// The packed column x2 = 0 of an FP32 spectrum (the kx = 0 and kx = N/2
// planes, A + iB) into bins: warp w of CTA b takes the row kz of iz = b W + w
// and rings j = |ky|, unpacking each slot with its partner at (-z, -y); the
// kx = 0 and kx = N/2 modes are two ring lines (n^2 = kz^2 + j^2 and
// kz^2 + (N/2)^2 + j^2).  The CTA's warp sums go to partials[slot0 + b].
constexpr int kPlaneBinWarps = 8;
template <int N>
__global__ void __launch_bounds__(kPlaneBinWarps * 32)
k_bin_plane0(const cx<float>* __restrict__ spec, int nk, const int* __restrict__ thr, float inv_lr,
             double* __restrict__ partials, int slot0) {
  constexpr int M = N / 2, J = N / 2, ER = J / 32;
  static_assert(J % 32 == 0, "rings per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* acc_all = reinterpret_cast<float2*>(smem_raw);   // [kPlaneBinWarps][nk] float pairs
  for (int i = threadIdx.x; i < kPlaneBinWarps * nk; i += blockDim.x) acc_all[i] = make_float2(0.0f, 0.0f);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int iz = blockIdx.x * kPlaneBinWarps + warp;
  if (iz < N) {
    const int kz = signed_freq(iz, N);
    const int pz = partner_index(iz, N);
    auto unpack = [&](int iy, float& pa, float& pb) {
      const cx<float> f = spec[((int64_t)iz * N + iy) * M];
      const cx<float> g = spec[((int64_t)pz * N + partner_index(iy, N)) * M];
      const float ax = 0.5f * (f.x + g.x), ay = 0.5f * (f.y - g.y);
      const float bx = 0.5f * (f.y + g.y), by = -0.5f * (f.x - g.x);
      pa = ax * ax + ay * ay;
      pb = bx * bx + by * by;
    };
    float ra[ER], rb[ER];
#pragma unroll
    for (int i = 0; i < ER; ++i) {
      const int j = lane * ER + i;   // j < J
      float a1, b1;
      unpack(j, a1, b1);
      if (j > 0) {
        float a2, b2;
        unpack(N - j, a2, b2);
        a1 += a2;
        b1 += b2;
      }
      ra[i] = (kz == 0 && j == 0) ? 0.0f : a1;   // the mean carries no power
      rb[i] = b1;
    }
    float ea = 0.0f, eb = 0.0f;
    if (lane == 31) unpack(J, ea, eb);           // ky = N/2: one mode
    float2* acc = acc_all + warp * nk;
    bin_rings_warp<ER>(ra, kz * kz, true, kz * kz + J * J, ea, thr, nk, inv_lr, acc);
    bin_rings_warp<ER>(rb, kz * kz + M * M, true, kz * kz + M * M + J * J, eb, thr, nk, inv_lr, acc);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kPlaneBinWarps; ++w) sum += (double)acc_all[w * nk + i].x + (double)acc_all[w * nk + i].y;
    partials[(int64_t)(slot0 + blockIdx.x) * nk + i] = sum;
  }
}

// One row's modes into the warp's accumulator acc (see above).  f: this
// lane's E modes (power sums only), g: lane 0's partner slot.
template <typename T, bool LATTICE>
__device__ __forceinline__ void bin_row(const cx<T> (&f)[kBinLaneMax], cx<T> g, int base2, int m, int E, int lane,
                                        const int* Ts, int nk, float inv_lr, double kf, double* acc) {
  using A = typename std::conditional<LATTICE, double, T>::type;   // run / segment sums
  const unsigned full = 0xffffffffu;
  const int xb = lane * E;
  auto add0 = [&](int b, A v) {
    if constexpr (kBinPair<T, LATTICE>) pair_add(reinterpret_cast<float2*>(acc) + b, (float)v);
    else acc[b] += (double)v;
  };
  // runs of this lane's modes
  int bF = -1, bL = -1, tnext = 0;
  bool multi = false;
  A sF0 = 0, sF1 = 0, c0 = 0, c1 = 0;
#pragma unroll
  for (int i = 0; i < kBinLaneMax; ++i) {
    const int x2 = xb + i;
    const int n2 = base2 + x2 * x2;
    if (i < E && x2 < m && n2 > 0) {
      A v0, v1 = 0;
      if constexpr (LATTICE) {
        v0 = x2 == 0 ? 1.0 : 2.0;
        v1 = v0 * kf * sqrt((double)n2);
      } else if (x2 == 0) {
        const T ax = (T)0.5 * (f[i].x + g.x), ay = (T)0.5 * (f[i].y - g.y);
        v0 = ax * ax + ay * ay;
      } else {
        v0 = (T)2 * (f[i].x * f[i].x + f[i].y * f[i].y);
      }
      if (bL < 0) {
        const int b0 = bin_of_n2(n2, Ts, nk, inv_lr);   // >= 0 for every 0 < n^2 <= 3 N^2 / 4
        if (b0 >= 0) {
          bL = bF = b0;
          tnext = Ts[b0 + 1];
        } else {
          v0 = v1 = 0;
        }
      } else if (n2 >= tnext) {
        if (!multi) {          // the first run waits for the lane combine
          sF0 = c0;
          sF1 = c1;
          multi = true;
        } else {               // an inner run: the whole bin of this row
          add0(bL, c0);
          if constexpr (LATTICE) acc[nk + bL] += (double)c1;
        }
        c0 = c1 = 0;
        do {
          ++bL;
          tnext = Ts[bL + 1];
        } while (n2 >= tnext);
      }
      c0 += v0;
      c1 += v1;
    }
  }
  // join the boundary runs across lanes: element (key, sums, open), where a
  // single-run lane is open (its run continues the previous lane's)
  int k = bL;
  bool open = !multi && bL >= 0;
  A s0 = c0, s1 = c1;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int pk = __shfl_up_sync(full, k, off);
    const A p0 = __shfl_up_sync(full, s0, off);
    A p1 = 0;
    if constexpr (LATTICE) p1 = __shfl_up_sync(full, s1, off);
    const bool popen = __shfl_up_sync(full, (int)open, off) != 0;
    if (lane >= off && open && pk == k) {
      s0 += p0;
      if constexpr (LATTICE) s1 += p1;
      open = popen;
    }
  }
  // segment ending in the previous lane, and the first bin of the next lane
  const int qk = __shfl_up_sync(full, k, 1);
  const A q0 = __shfl_up_sync(full, s0, 1);
  A q1 = 0;
  if constexpr (LATTICE) q1 = __shfl_up_sync(full, s1, 1);
  const int nextF = __shfl_down_sync(full, bF, 1);
  __syncwarp();
  if (multi) {   // first run closes the incoming segment of its bin
    const bool join = lane > 0 && qk == bF;
    add0(bF, sF0 + (join ? q0 : (A)0));
    if constexpr (LATTICE) acc[nk + bF] += (double)(sF1 + (join ? q1 : (A)0));
  }
  __syncwarp();
  if (k >= 0 && (lane == 31 || nextF != k)) {   // the segment ends here
    add0(k, s0);
    if constexpr (LATTICE) acc[nk + k] += (double)s1;
  }
  __syncwarp();
  if (lane == 0) {   // the kx = N/2 mode of the packed slot, weight 1
    const int n2b = base2 + m * m;
    const int bb = bin_of_n2(n2b, Ts, nk, inv_lr);
    if (bb >= 0) {
      if constexpr (LATTICE) {
        acc[bb] += 1.0;
        acc[nk + bb] += kf * sqrt((double)n2b);
      } else {
        const T bx = (T)0.5 * (f[0].y + g.y), by = (T)-0.5 * (f[0].x - g.x);
        add0(bb, bx * bx + by * by);
      }
    }
  }
  __syncwarp();
}

template <typename T, bool LATTICE>
__device__ __forceinline__ void bin_flush_partials(const double* all, int nk, double* partials, int64_t slot) {
  constexpr int NV = LATTICE ? 2 : 1;
  __syncthreads();
  for (int i = threadIdx.x; i < NV * nk; i += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int wi = 0; wi < kBinWarps; ++wi) {
      if constexpr (kBinPair<T, LATTICE>) {
        const float2 p = reinterpret_cast<const float2*>(all)[wi * NV * nk + i];
        sum += (double)p.x + (double)p.y;
      } else {
        sum += all[wi * NV * nk + i];
      }
    }
    partials[slot * NV * nk + i] = sum;
  }
}

// Rows read by each lane from global memory (lattice sums, and grids whose
// lane segments are not whole 16-byte units).
// Body: rows row0 + warp, row0 + warp + row_step, ... below row1 into the
// per-warp accumulators, then their sum to partials[slot].
template <typename T, bool LATTICE>
__device__ __forceinline__ void bin_power_rows(const cx<T>* __restrict__ spec, int n, int nk,
                                               const int* __restrict__ thr, float inv_lr, double kf,
                                               double* __restrict__ partials, int row0, int row1, int row_step,
                                               int64_t slot) {
  constexpr int NV = LATTICE ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* all = reinterpret_cast<double*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = all + warp * NV * nk;
  int* Ts = reinterpret_cast<int*>(all + kBinWarps * NV * nk);
  for (int i = threadIdx.x; i < kBinWarps * NV * nk; i += blockDim.x) all[i] = 0.0;
  for (int i = threadIdx.x; i <= nk; i += blockDim.x) Ts[i] = thr[i];
  __syncthreads();
  const int m = n / 2;
  const int E = (m + 31) >> 5;
  const int xb = lane * E;
  for (int row = row0 + warp; row < row1; row += row_step) {
    const int iz = row / n, iy = row - (row / n) * n;
    const int kz = signed_freq(iz, n), ky = signed_freq(iy, n);
    const cx<T>* r = spec + (int64_t)row * m;
    cx<T> g = {(T)0, (T)0};   // lane 0: the packed slot of the partner row (-z, -y)
    cx<T> f[kBinLaneMax];
    if constexpr (!LATTICE) {
      if (lane == 0) g = spec[((int64_t)partner_index(iz, n) * n + partner_index(iy, n)) * m];
#pragma unroll
      for (int i = 0; i < kBinLaneMax; ++i)
        if (i < E && xb + i < m) f[i] = r[xb + i];
    }
    bin_row<T, LATTICE>(f, g, kz * kz + ky * ky, m, E, lane, Ts, nk, inv_lr, kf, acc);
  }
  bin_flush_partials<T, LATTICE>(all, nk, partials, slot);
}

template <typename T, bool LATTICE>
__global__ void __launch_bounds__(kBinWarps * 32)
k_bin_power(const cx<T>* __restrict__ spec, int n, int nk, const int* __restrict__ thr, float inv_lr,
            double kf, double* __restrict__ partials) {
  bin_power_rows<T, LATTICE>(spec, n, nk, thr, inv_lr, kf, partials, blockIdx.x * kBinWarps, n * n,
                             gridDim.x * kBinWarps, blockIdx.x);
}

// bin_row for the staged power sums: E (compile time) modes per lane, all
// inside the row; the lane's first bin is found once, the run keys carry
// their open flag in bit 0 so the lane scan moves two words per step.  The
// kx = N/2 mode of the packed slot (n^2 = base2 + M^2, weight 1) is lane 31's
// last mode, so it joins the runs instead of a separate add.
template <typename T, int E>
__device__ __forceinline__ void bin_row_staged(const cx<T> (&f)[kBinLaneMax], cx<T> g, int base2, int lane,
                                               const int* Ts, int nk, float inv_lr, double* acc) {
  constexpr int M = 32 * E;
  auto add0 = [&](int b, T v) {
    if constexpr (sizeof(T) == 4) pair_add(reinterpret_cast<float2*>(acc) + b, (float)v);
    else acc[b] += (double)v;
  };
  const unsigned full = 0xffffffffu;
  const int xb = lane * E;
  // lane 0 unpacks the slot: A (kx = 0) stays, B (kx = N/2) goes to lane 31
  const T ax = (T)0.5 * (f[0].x + g.x), ay = (T)0.5 * (f[0].y - g.y);
  const T bx = (T)0.5 * (f[0].y + g.y), by = (T)-0.5 * (f[0].x - g.x);
  const T vB = __shfl_sync(full, bx * bx + by * by, 0);
  int n2 = base2 + xb * xb;
  int bL = bin_of_n2(n2 > 0 ? n2 : 1, Ts, nk, inv_lr);   // n^2 = 0 (the mean) adds nothing
  const int bF = bL;
  int tnext = Ts[bL + 1];
  bool multi = false;
  T sF = 0, c = 0;
  auto mode = [&](int n2m, T v) {
    if (n2m >= tnext) {
      if (!multi) {          // the first run waits for the lane combine
        sF = c;
        multi = true;
      } else {               // an inner run: the whole bin of this row
        add0(bL, c);
      }
      c = 0;
      do {
        ++bL;
        tnext = Ts[bL + 1];
      } while (n2m >= tnext);
    }
    c += v;
  };
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int x2 = xb + i;
    if (i > 0) n2 = base2 + x2 * x2;
    T v;
    if (i == 0 && lane == 0) v = n2 > 0 ? ax * ax + ay * ay : (T)0;   // kx = 0 mode, weight 1
    else v = (T)2 * (f[i].x * f[i].x + f[i].y * f[i].y);
    mode(n2, v);
  }
  if (lane == 31) mode(base2 + M * M, vB);
  int kk = (bL << 1) | (multi ? 0 : 1);   // key, open (a single-run lane continues the previous one)
  T s0 = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int pkk = __shfl_up_sync(full, kk, off);
    const T p0 = __shfl_up_sync(full, s0, off);
    if (lane >= off && (kk & 1) && (pkk >> 1) == (kk >> 1)) {
      s0 += p0;
      kk = (kk & ~1) | (pkk & 1);
    }
  }
  const int k = kk >> 1;
  const int qk = __shfl_up_sync(full, k, 1);
  const T q0 = __shfl_up_sync(full, s0, 1);
  const int nextF = __shfl_down_sync(full, bF, 1);
  __syncwarp();
  if (multi) add0(bF, sF + ((lane > 0 && qk == bF) ? q0 : (T)0));
  __syncwarp();
  if (lane == 31 || nextF != k) add0(k, s0);
  __syncwarp();
}

// FP32 power sums with the rows staged by TMA: each warp runs a
// kBinStages-deep ring of row buffers in shared memory (two: 5 CTAs per SM
// at 1024^3, where three allowed 3 and the combine went short of warps).  A tensor map views
// the spectrum as [rows][32 lanes][E modes] (8-byte elements); one 3-D copy
// brings a whole row, swizzled with the span equal to a lane's segment
// (E = 4, 8, 16: 32-, 64-, 128-byte swizzle; E = 2: none), so lane L reading
// its own E modes as 16-byte units hits a different bank group from its
// neighbours.  Each row buffer holds 4 KB whatever E.  A 16-byte bulk copy
// brings the partner row's packed slot.  The copies of row r + kBinStages
// steps are issued as soon as row r is in registers.  Waits are bounded: on a
// timeout the kernel records PM_ERR_TIMEOUT, waits (bounded) for its own
// copies still in flight and stops.
constexpr int kBinStages = 2;

// Bytes of one staged row buffer: 32 lines of 128 bytes (a whole number of
// swizzle atoms for every span), also when the row itself is smaller.
__host__ __device__ constexpr int bin_stage_row_bytes(int) { return 32 * 128; }
// Shared memory of k_bin_power_tma: accumulators and thresholds (rounded up
// to 1024 bytes), the warps' row rings, partner slots, mbarriers.
__host__ __device__ constexpr size_t bin_tma_head(int nk) {
  return ((size_t)kBinWarps * nk * sizeof(double) + (size_t)(nk + 1) * sizeof(int) + 1023) & ~(size_t)1023;
}
__host__ __device__ constexpr size_t bin_tma_smem(int nk, int E) {
  return bin_tma_head(nk) + (size_t)kBinWarps * kBinStages * (bin_stage_row_bytes(E) + 16 + sizeof(uint64_t)) +
         1024;   // slack to align the dynamic base to 1024 bytes
}

// Byte offset of linear offset lin under the TMA swizzle whose span is the
// E * 8-byte lane segment: 16-byte unit bits [4, 4 + s) XOR address bits
// [7, 7 + s), s = log2(E * 8 / 16).
template <int E>
__device__ __forceinline__ int swizzle_lane(int lin) {
  constexpr int mask = E == 16 ? 0x70 : E == 8 ? 0x30 : E == 4 ? 0x10 : 0;
  return lin ^ ((lin >> 3) & mask);
}

template <int E>
__global__ void __launch_bounds__(kBinWarps * 32)
k_bin_power_tma(const __grid_constant__ CUtensorMap map, const cx<float>* __restrict__ spec, int n, int nk,
                const int* __restrict__ thr, float inv_lr, double* __restrict__ partials, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
  double* all = reinterpret_cast<double*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = all + warp * nk;
  int* Ts = reinterpret_cast<int*>(all + kBinWarps * nk);
  constexpr int RB = bin_stage_row_bytes(E);
  const size_t head = bin_tma_head(nk);
  unsigned char* rows_s = smem_raw + head + (size_t)warp * kBinStages * RB;
  unsigned char* part_s = smem_raw + head + (size_t)kBinWarps * kBinStages * RB + (size_t)warp * kBinStages * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + head + (size_t)kBinWarps * kBinStages * (RB + 16)) +
                   warp * kBinStages;
  for (int i = threadIdx.x; i < kBinWarps * nk; i += blockDim.x) all[i] = 0.0;
  for (int i = threadIdx.x; i <= nk; i += blockDim.x) Ts[i] = thr[i];
  if (lane == 0) {
    for (int st = 0; st < kBinStages; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned full = 0xffffffffu;
  constexpr int N = 64 * E, M = 32 * E;            // n == N
  const int rows = N * N;
  const int step = gridDim.x * kBinWarps;
  const int row0 = blockIdx.x * kBinWarps + warp;
  auto issue = [&](int row, int st) {   // lane 0
    mbar_expect_tx(&bars[st], (uint32_t)(32 * E * 8 + 16));
    tma_load_3d(rows_s + (size_t)st * RB, &map, &bars[st], 0, 0, row);
    const int iz = row / N, iy = row % N;
    bulk_load(part_s + st * 16, spec + ((int64_t)partner_index(iz, N) * N + partner_index(iy, N)) * M, 16u,
              &bars[st]);
  };
  if (lane == 0)
    for (int st = 0; st < kBinStages; ++st)
      if (row0 + st * step < rows) issue(row0 + st * step, st);
  int k = 0;
  for (int row = row0; row < rows; row += step, ++k) {
    const int st = k % kBinStages;
    const uint32_t parity = (uint32_t)((k / kBinStages) & 1);
    const bool ok = mbar_wait_bounded(&bars[st], parity);
    if (!__all_sync(full, ok)) {
      if (lane == 0) {
        atomicCAS(status, 0, PM_ERR_TIMEOUT);
        // this warp's copies still in flight: rows row .. row + (kBinStages - 1) steps
        for (int j = 0; j < kBinStages; ++j)
          if (row + j * step < rows)
            mbar_wait_bounded(&bars[(k + j) % kBinStages], (uint32_t)(((k + j) / kBinStages) & 1));
      }
      __syncwarp();
      break;
    }
    const unsigned char* buf = rows_s + (size_t)st * RB;
    cx<float> f[kBinLaneMax];
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(buf + swizzle_lane<E>(lane * E * 8 + 16 * j));
      f[2 * j] = {v.x, v.y};
      f[2 * j + 1] = {v.z, v.w};
    }
    const cx<float> g = *reinterpret_cast<const cx<float>*>(part_s + st * 16);
    fence_proxy_async_shared();   // these reads come before the buffer's next copy
    __syncwarp();
    if (lane == 0 && row + kBinStages * step < rows) issue(row + kBinStages * step, st);
    const int iz = row / N, iy = row % N;
    const int kz = signed_freq(iz, N), ky = signed_freq(iy, N);
    bin_row_staged<float, E>(f, g, kz * kz + ky * ky, lane, Ts, nk, inv_lr, acc);
  }
  bin_flush_partials<float, false>(all, nk, partials, blockIdx.x);
}

// ---------------------------------------------------------------------------
// a5 on the packed column x2 = 0: its slot holds A + i B, the kx = 0 and
// kx = N/2 plane spectra, whose Green factors differ.  Unpack with the
// partner at (-ky, -kz), multiply each by its G(n^2) (and deconvolution), and
// repack P = G_A A + i G_B B into plane0[ky][kz] for k_fft_z_inv_green.
// ---------------------------------------------------------------------------
// Body: plane0 entries idx0, idx0 + step, ... below idx1.
template <typename T>
__device__ __forceinline__ void green_plane0_range(const cx<T>* __restrict__ spec, cx<T>* __restrict__ plane0, int n,
                                                   const T* __restrict__ gtab, const T* __restrict__ wtab,
                                                   const float* __restrict__ fac, float fac_inv_du, float coeff,
                                                   int idx0, int idx1, int step) {
  // G(n^2): the FP64 table, or (FP32) coeff fac(u) / n^2 from the fac table as
  // in the inverse z passes; G(0) = 0
  auto green = [&](int n2) -> T {
    if constexpr (sizeof(T) == 4) {
      if (n2 == 0) return (T)0;
      const float tt = 0.5f * __logf((float)n2) * fac_inv_du;
      const int j = min((int)tt, kFacTableDev - 2);
      const float fr = tt - (float)j;
      return (T)(coeff * (fac[j] + fr * (fac[j + 1] - fac[j])) / (float)n2);
    } else {
      return gtab[n2];
    }
  };
  const int m = n / 2;
  for (int idx = idx0; idx < idx1; idx += step) {
    const int iy = idx / n, iz = idx - (idx / n) * n;    // plane0 layout [ky][kz]
    const int ky = signed_freq(iy, n), kz = signed_freq(iz, n);
    const int jy = partner_index(iy, n), jz = partner_index(iz, n);
    const cx<T> f = spec[((int64_t)iz * n + iy) * m];
    const cx<T> h = spec[((int64_t)jz * n + jy) * m];
    const cx<T> A = {(T)0.5 * (f.x + h.x), (T)0.5 * (f.y - h.y)};
    const cx<T> B = {(T)0.5 * (f.y + h.y), (T)-0.5 * (f.x - h.x)};
    const int n2a = ky * ky + kz * kz;
    T ga = green(n2a), gb = green(n2a + m * m);
    if (wtab) {
      const T wyz = wtab[iy] * wtab[iz];
      ga *= wtab[0] * wyz;
      gb *= wtab[m] * wyz;
    }
    plane0[idx] = {ga * A.x - gb * B.y, ga * A.y + gb * B.x};   // G_A A + i G_B B
  }
}

template <typename T>
__global__ void k_green_plane0(const cx<T>* __restrict__ spec, cx<T>* __restrict__ plane0, int n,
                               const T* __restrict__ gtab, const T* __restrict__ wtab, const float* __restrict__ fac,
                               float fac_inv_du, float coeff) {
  green_plane0_range<T>(spec, plane0, n, gtab, wtab, fac, fac_inv_du, coeff, blockIdx.x * blockDim.x + threadIdx.x,
                        n * n, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// a7: CIC interpolation of the three real force grids (same quantised
// weights as the deposit) and the kick u += acc * K.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_interp_kick(const void* __restrict__ pos, int64_t np, int n, double delta,
                              const T* __restrict__ grids, int64_t field_stride, T* __restrict__ vel,
                              T kick, T* __restrict__ acc_out, int* status) {
  constexpr int U = kInterpBatch;
  // a warp takes U x 32 consecutive particles (its U loads per lane 32 apart),
  // so the force rows one warp gathers stay close together
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * U;
  for (int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * U + (threadIdx.x & 31); p0 < np;
       p0 += stride) {
    typename Quant<T>::Raw raw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * 32;
      if (p < np) raw[u] = Quant<T>::load(pos, np, p);
    }
    // gather all corners of all U particles before the arithmetic
    T g[U][3][8];
    T f[U][6];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int c[3], w[3];
      ok[u] = p0 + u * 32 < np && Quant<T>::get(raw[u], n, delta, c, w, status);
      if (!ok[u]) continue;
      const T inv = (T)1.0 / (T)kWeightOne;
      f[u][1] = (T)w[0] * inv;
      f[u][3] = (T)w[1] * inv;
      f[u][5] = (T)w[2] * inv;
      f[u][0] = (T)1 - f[u][1];
      f[u][2] = (T)1 - f[u][3];
      f[u][4] = (T)1 - f[u][5];
      const int x1 = c[0] + 1 == n ? 0 : c[0] + 1;
      const int y1 = c[1] + 1 == n ? 0 : c[1] + 1;
      const int z1 = c[2] + 1 == n ? 0 : c[2] + 1;
      const int64_t r[4] = {((int64_t)c[2] * n + c[1]) * n, ((int64_t)c[2] * n + y1) * n,
                            ((int64_t)z1 * n + c[1]) * n, ((int64_t)z1 * n + y1) * n};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T* gd = grids + d * field_stride;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          g[u][d][2 * q] = gd[r[q] + c[0]];
          g[u][d][2 * q + 1] = gd[r[q] + x1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int64_t p = p0 + u * 32;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T v00 = f[u][0] * g[u][d][0] + f[u][1] * g[u][d][1];   // (y0, z0)
        const T v01 = f[u][0] * g[u][d][2] + f[u][1] * g[u][d][3];   // (y1, z0)
        const T v10 = f[u][0] * g[u][d][4] + f[u][1] * g[u][d][5];   // (y0, z1)
        const T v11 = f[u][0] * g[u][d][6] + f[u][1] * g[u][d][7];   // (y1, z1)
        const T a = f[u][4] * (f[u][2] * v00 + f[u][3] * v01) + f[u][5] * (f[u][2] * v10 + f[u][3] * v11);
        vel[d * np + p] += a * kick;
        if (acc_out) acc_out[d * np + p] = a;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// a6-a7 with the gradient taken in real space.  The 4-point central
// difference whose Fourier multiplier is -i D(k) (D(k) = [8 sin(k d) -
// sin(2 k d)] / (6 d), d the cell size) is, on the periodic grid,
//   (S f)(x) = [f(x-2) - 8 f(x-1) + 8 f(x+1) - f(x+2)] / (12 d),
// so acc = -S phi on the potential grid equals the inverse transform of
// -i D G delta in exact arithmetic (the multiplier and the stencil both
// vanish on the Nyquist index).  The gather applies S at the particle's eight
// CIC corners; along an axis the corners c and c + 1 see the potential at
// c - 2 .. c + 3 with the folded weights
//   e_j = w0 s(j - 2) + w1 s(j - 3),  s(-2..2) = (1, -8, 0, 8, -1),
// so each particle reads 56 potential values (four 6-point runs along x,
// eight 4-point runs along y and along z) instead of 3 x 8 force values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_near(int c, int d, int n) {
  int v = c + d;   // d in [-2, 3], c in [0, n), n >= 16
  if ((n & (n - 1)) == 0) return v & (n - 1);
  v = v < 0 ? v + n : v;
  return v >= n ? v - n : v;
}

template <typename T>
__device__ __forceinline__ void fold_weights(T f0, T f1, T (&e)[6]) {
  e[0] = f0;
  e[1] = (T)-8 * f0 + f1;
  e[2] = (T)-8 * f1;
  e[3] = (T)8 * f0;
  e[4] = -f0 + (T)8 * f1;
  e[5] = -f1;
}

// -S phi at one particle (cell c, 16-bit weights w), before the -1/(12 d)
// scale: the CIC sum of the 4-point stencil at its 8 corners (see above).
template <typename T>
__device__ __forceinline__ void fd_stencil(const T* __restrict__ phi, int n, const int (&c)[3], const int (&w)[3],
                                           T (&a)[3]) {
  const T inv = (T)1.0 / (T)kWeightOne;
  int xs[6], ys[6], zs[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    xs[j] = wrap_near(c[0], j - 2, n);
    ys[j] = wrap_near(c[1], j - 2, n);
    zs[j] = wrap_near(c[2], j - 2, n);
  }
  // (y, z) row starts; indices < 2^30 for n <= 1024
  auto row = [&](int y, int z) { return ((uint32_t)z * (uint32_t)n + (uint32_t)y) * (uint32_t)n; };
  T px[2][2][6];   // [dz][dy][x0-2 .. x0+3]
  T py[2][2][4];   // [dz][dx][y0-2, y0-1, y0+2, y0+3]
  T pz[2][2][4];   // [dy][dx][z0-2, z0-1, z0+2, z0+3]
  constexpr int kFar[4] = {0, 1, 4, 5};
  // FP32 x runs away from the row ends: aligned 8-byte loads from a = (x0 - 2)
  // rounded down to even cover x0 - 2 .. x0 + 3 (three loads, a fourth when
  // x0 is odd), picked by o = (x0 - 2) & 1
  const int a2 = (c[0] - 2) & ~1;
  if (sizeof(T) == 4 && c[0] >= 2 && a2 + 8 <= n) {
    const int o = (c[0] - 2) & 1;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float2* r2 = reinterpret_cast<const float2*>(phi + row(ys[2 + dy], zs[2 + dz]) + a2);
        const float2 q0 = r2[0], q1 = r2[1], q2 = r2[2];
        const float2 q3 = o ? r2[3] : make_float2(0.0f, 0.0f);
        const float w8[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
#pragma unroll
        for (int j = 0; j < 6; ++j) px[dz][dy][j] = (T)(o ? w8[j + 1] : w8[j]);
      }
  } else {
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const T* r = phi + row(ys[2 + dy], zs[2 + dz]);
#pragma unroll
        for (int j = 0; j < 6; ++j) px[dz][dy][j] = r[xs[j]];
      }
  }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T* r = phi + row(ys[kFar[q]], zs[2 + dz]);
      py[dz][0][q] = r[xs[2]];
      py[dz][1][q] = r[xs[3]];
    }
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T* r = phi + row(ys[2 + dy], zs[kFar[q]]);
      pz[dy][0][q] = r[xs[2]];
      pz[dy][1][q] = r[xs[3]];
    }
  T f[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d][1] = (T)w[d] * inv;
    f[d][0] = (T)1 - f[d][1];
  }
  T ex[6], ey[6], ez[6];
  fold_weights(f[0][0], f[0][1], ex);
  fold_weights(f[1][0], f[1][1], ey);
  fold_weights(f[2][0], f[2][1], ez);
  a[0] = a[1] = a[2] = (T)0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      T sx = (T)0;
#pragma unroll
      for (int j = 0; j < 6; ++j) sx += ex[j] * px[dz][dy][j];
      a[0] += f[1][dy] * f[2][dz] * sx;
    }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const T sy = ey[0] * py[dz][dx][0] + ey[1] * py[dz][dx][1] + ey[2] * px[dz][0][2 + dx] +
                   ey[3] * px[dz][1][2 + dx] + ey[4] * py[dz][dx][2] + ey[5] * py[dz][dx][3];
      a[1] += f[0][dx] * f[2][dz] * sy;
    }
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const T sz = ez[0] * pz[dy][dx][0] + ez[1] * pz[dy][dx][1] + ez[2] * px[0][dy][2 + dx] +
                   ez[3] * px[1][dy][2 + dx] + ez[4] * pz[dy][dx][2] + ez[5] * pz[dy][dx][3];
      a[2] += f[0][dx] * f[1][dy] * sz;
    }
}

// Work order: CTA b takes the kGatherChunk x kGatherTPB consecutive particles
// from b kGatherChunk kGatherTPB on (its threads kGatherTPB apart, each thread
// kGatherChunk particles), and CTAs are dispatched in index order, so the
// particles in flight at any time form one narrow window of the array: for
// particles near storage (lattice) order the potential rows they read stay in
// L2 between neighbouring CTAs.  (A grid-stride loop over the whole array lets
// warps drift apart by hundreds of particle planes, and the potential was
// re-read from DRAM: 1.5x the compulsory bytes, and 4x the time for clustered
// inputs, measured on GB300.)
constexpr int kGatherTPB = 64;
constexpr int kGatherChunk = 8;

// Body: chunk `chunk` of kGatherTPB x kGatherChunk particles (blockDim = kGatherTPB).
template <typename T>
__device__ __forceinline__ void interp_fd_chunk(const void* __restrict__ pos, int64_t np, int n, double delta,
                                                const T* __restrict__ phi, T* __restrict__ vel, T kick,
                                                T* __restrict__ acc_out, int* status, int64_t chunk) {
  const T scale = (T)(-1.0 / (12.0 * delta));   // acc = -S phi
  const int64_t base = chunk * kGatherTPB * kGatherChunk + threadIdx.x;
  // the next particle's position words are fetched while this one's
  // potential values are in flight (one memory round trip per particle)
  typename Quant<T>::Raw next;
  if (base < np) next = Quant<T>::load(pos, np, base);
#pragma unroll 1
  for (int u = 0; u < kGatherChunk; ++u) {
    const int64_t p = base + (int64_t)u * kGatherTPB;
    if (p >= np) break;
    const typename Quant<T>::Raw raw = next;
    if (u + 1 < kGatherChunk && p + kGatherTPB < np) next = Quant<T>::load(pos, np, p + kGatherTPB);
    const T u0 = vel[p], u1 = vel[np + p], u2 = vel[2 * np + p];
    int c[3], w[3];
    if (!Quant<T>::get(raw, n, delta, c, w, status)) continue;
    T a[3];
    fd_stencil<T>(phi, n, c, w, a);
    const T uu[3] = {u0, u1, u2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T ad = a[d] * scale;
      vel[d * np + p] = uu[d] + ad * kick;
      if (acc_out) acc_out[d * np + p] = ad;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kGatherTPB, sizeof(T) == 4 ? 12 : 8)
k_interp_kick_fd(const void* __restrict__ pos, int64_t np, int n, double delta, const T* __restrict__ phi,
                 T* __restrict__ vel, T kick, T* __restrict__ acc_out, int* status) {
  interp_fd_chunk<T>(pos, np, n, delta, phi, vel, kick, acc_out, status, blockIdx.x);
}

// The same gather in the row order of the deposit's sort: one warp per grid
// row (z, y), its lanes over the row's records (x cell and weights; y and z
// are the row's) and perm[] giving each record's particle for the velocity
// update.  Particles far from their storage order (clustered inputs) then
// still read neighbouring potential rows warp by warp.  The arithmetic is
// fd_stencil's: forces bit-identical to the particle-order gather.
// Rows in index order: CTA b takes rows b kRowsPerCta .. (b + 1) kRowsPerCta - 1
// (its warps round robin), dispatched in order as the particle-order gather.
constexpr int kRowsPerCta = 8;

template <typename T>
__global__ void __launch_bounds__(kGatherTPB, sizeof(T) == 4 ? 10 : 8)
k_interp_rows_fd(const unsigned long long* __restrict__ rec, const int* __restrict__ row_start,
                 const int* __restrict__ perm, int64_t np, int n, double delta, const T* __restrict__ phi,
                 T* __restrict__ vel, T kick, T* __restrict__ acc_out) {
  const T scale = (T)(-1.0 / (12.0 * delta));
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int rows = n * n;
  const int r0 = blockIdx.x * kRowsPerCta;
  for (int row = r0 + (threadIdx.x >> 5); row < r0 + kRowsPerCta && row < rows; row += wpb) {
    const int beg = row_start[row], end = row_start[row + 1];
    const int cz = row / n, cy = row - cz * n;
    for (int i = beg + lane; i < end; i += 32) {
      const unsigned long long r = rec[i];
      const int64_t p = perm[i];
      const T u0 = vel[p], u1 = vel[np + p], u2 = vel[2 * np + p];
      const int c[3] = {(int)(r >> 48) & 0x7ff, cy, cz};
      const int w[3] = {(int)(r & 0xffffu), (int)((r >> 16) & 0xffffu), (int)((r >> 32) & 0xffffu)};
      T a[3];
      fd_stencil<T>(phi, n, c, w, a);
      const T u[3] = {u0, u1, u2};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T ad = a[d] * scale;
        vel[d * np + p] = u[d] + ad * kick;
        if (acc_out) acc_out[d * np + p] = ad;
      }
    }
  }
}

// The row-order gather without its scattered velocity update (clustered
// particles, far from their storage order, make the update through perm[] a
// random read and write of six words a particle): the forces of the sorted
// records are written by sorted slot, four values a slot (one 16- or 32-byte
// store), and k_kick_inv then walks the particles in storage order, reading
// each one's force through its slot inv[p] (one random 16- or 32-byte read)
// and updating its velocity with coalesced accesses.  fd_stencil's arithmetic
// and the same update expression: bit-identical to the particle-order gather.
// Work order: the sorted records in contiguous chunks of kGatherTPB x
// kGatherChunk (a CTA's threads kGatherTPB apart, as the particle-order
// gather), CTAs dispatched in index order.  The CTA finds the row of its first
// record by bisection of row_start; each thread then advances its row as its
// records advance (rows are sorted), so empty rows cost nothing.
template <typename T>
__global__ void __launch_bounds__(kGatherTPB, sizeof(T) == 4 ? 12 : 8)
k_interp_rows_acc(const unsigned long long* __restrict__ rec, const int* __restrict__ row_start, int n,
                  double delta, const T* __restrict__ phi, T* __restrict__ accs) {
  __shared__ int s_row;
  const T scale = (T)(-1.0 / (12.0 * delta));
  const int rows = n * n;
  const int nrec = row_start[rows];                 // the sorted (valid) records
  const int64_t i0 = (int64_t)blockIdx.x * kGatherTPB * kGatherChunk;
  if (i0 >= nrec) return;
  if (threadIdx.x == 0) {
    int lo = 0, hi = rows;                          // row_start[lo] <= i0 < row_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (row_start[mid] <= i0) lo = mid; else hi = mid;
    }
    s_row = lo;
  }
  __syncthreads();
  int r = s_row;
#pragma unroll 1
  for (int u = 0; u < kGatherChunk; ++u) {
    const int64_t i = i0 + threadIdx.x + (int64_t)u * kGatherTPB;
    if (i >= nrec) break;
    while (row_start[r + 1] <= i) ++r;              // r + 1 <= rows: i < row_start[rows]
    const int cz = r / n, cy = r - cz * n;
    const unsigned long long rr = rec[i];
    const int c[3] = {(int)(rr >> 48) & 0x7ff, cy, cz};
    const int w[3] = {(int)(rr & 0xffffu), (int)((rr >> 16) & 0xffffu), (int)((rr >> 32) & 0xffffu)};
    T a[3];
    fd_stencil<T>(phi, n, c, w, a);
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(accs)[i] = make_float4(a[0] * scale, a[1] * scale, a[2] * scale, 0.0f);
    } else {
      double2* q = reinterpret_cast<double2*>(accs) + 2 * i;
      q[0] = make_double2(a[0] * scale, a[1] * scale);
      q[1] = make_double2(a[2] * scale, 0.0);
    }
  }
}

template <typename T>
__global__ void k_kick_inv(const int* __restrict__ inv, const T* __restrict__ accs, int64_t np,
                           T* __restrict__ vel, T kick, T* __restrict__ acc_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
    const int slot = inv[p];
    if (slot < 0) continue;   // skipped by the sort (PM_ERR_RANGE recorded there)
    T ad[3];
    if constexpr (sizeof(T) == 4) {
      const float4 q = reinterpret_cast<const float4*>(accs)[slot];
      ad[0] = q.x;
      ad[1] = q.y;
      ad[2] = q.z;
    } else {
      const double2* q = reinterpret_cast<const double2*>(accs) + 2 * (int64_t)slot;
      const double2 q0 = q[0], q1 = q[1];
      ad[0] = q0.x;
      ad[1] = q0.y;
      ad[2] = q1.x;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      vel[d * np + p] = vel[d * np + p] + ad[d] * kick;
      if (acc_out) acc_out[d * np + p] = ad[d];
    }
  }
}

// Inspection: one component of acc = -S phi on the whole grid (real [N][N][N]).
template <typename T>
__global__ void k_fd_force_field(const T* __restrict__ phi, int n, int comp, double delta, T* __restrict__ out) {
  const T scale = (T)(-1.0 / (12.0 * delta));
  const int64_t total = (int64_t)n * n * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((int64_t)n * n));
    int idx[5];
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      const int xx = comp == 0 ? wrap_near(x, o, n) : x;
      const int yy = comp == 1 ? wrap_near(y, o, n) : y;
      const int zz = comp == 2 ? wrap_near(z, o, n) : z;
      idx[o + 2] = (zz * n + yy) * n + xx;
    }
    out[i] = scale * ((phi[idx[0]] - phi[idx[4]]) + (T)8 * (phi[idx[3]] - phi[idx[1]]));
  }
}

// ---------------------------------------------------------------------------
// Sec. 4.3 step (ii): particles moved to the next time step, x += u Delta s.
// Fixed IEEE roundings (no contraction into fused multiply-adds):
//   FP64  x' = x + (u ds), wrapped by one add or subtract of L (L itself -> 0)
//   FP32  d = u g, o' = o + d, k = floor(o'), o'' = o' - k (1 -> 0, k + 1),
//         cell = (cell + k) mod N,  g = Delta s / cell size in FP32
// A particle whose result is not finite (or whose FP32 offset is outside
// [0, 1) on entry) is left as it is and PM_ERR_RANGE is recorded.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_drift(void* __restrict__ pos, const T* __restrict__ vel, int64_t np, int n, double box,
                        double ds, float g, int* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
    bool ok = true;
    if constexpr (sizeof(T) == 8) {
      double* x = reinterpret_cast<double*>(pos);
      double xn[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double v = __dadd_rn(x[d * np + p], __dmul_rn((double)vel[d * np + p], ds));
        ok = ok && isfinite(v);
        if (v < 0.0) v = __dadd_rn(v, box);
        if (v >= box) v = __dsub_rn(v, box);
        if (v >= box) v = 0.0;
        xn[d] = v;
      }
      if (!ok) {
        set_status(status, PM_ERR_RANGE);
        continue;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d * np + p] = xn[d];
    } else {
      int32_t* q = reinterpret_cast<int32_t*>(pos);
      int cn[3];
      float on[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float o = __int_as_float(q[(3 + d) * np + p]);
        ok = ok && o >= 0.0f && o < 1.0f;
        const float o1 = __fadd_rn(o, __fmul_rn((float)vel[d * np + p], g));
        ok = ok && fabsf(o1) < 1.0e9f;          // finite, and the cell step fits an int
        const float k = floorf(o1);
        float o2 = __fsub_rn(o1, k);
        int kk = ok ? (int)k : 0;
        if (o2 >= 1.0f) {
          o2 = 0.0f;
          kk += 1;
        }
        cn[d] = wrap_index((long long)q[d * np + p] + kk, n);
        on[d] = o2;
      }
      if (!ok) {
        set_status(status, PM_ERR_RANGE);
        continue;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        q[d * np + p] = cn[d];
        q[(3 + d) * np + p] = __float_as_int(on[d]);
      }
    }
  }
}

// The FP32 drift four particles a thread with 16-byte loads and stores (npart
// a multiple of 4, so every row of the [6][np] words and [3][np] velocities
// starts 16-byte aligned); each particle follows k_drift's roundings exactly.
static __global__ void k_drift4(int32_t* __restrict__ q, const float* __restrict__ vel, int64_t np, int n, float g,
                         int* status) {
  const int64_t n4 = np >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    int cc[3][4], oo[3][4];
    float vv[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int4 c4 = reinterpret_cast<const int4*>(q + d * np)[i];
      const int4 o4 = reinterpret_cast<const int4*>(q + (3 + d) * np)[i];
      const float4 v4 = reinterpret_cast<const float4*>(vel + d * np)[i];
      cc[d][0] = c4.x; cc[d][1] = c4.y; cc[d][2] = c4.z; cc[d][3] = c4.w;
      oo[d][0] = o4.x; oo[d][1] = o4.y; oo[d][2] = o4.z; oo[d][3] = o4.w;
      vv[d][0] = v4.x; vv[d][1] = v4.y; vv[d][2] = v4.z; vv[d][3] = v4.w;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool ok = true;
      int cn[3], on[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float o = __int_as_float(oo[d][k]);
        ok = ok && o >= 0.0f && o < 1.0f;
        const float o1 = __fadd_rn(o, __fmul_rn(vv[d][k], g));
        ok = ok && fabsf(o1) < 1.0e9f;
        const float kf = floorf(o1);
        float o2 = __fsub_rn(o1, kf);
        int kk = ok ? (int)kf : 0;
        if (o2 >= 1.0f) {
          o2 = 0.0f;
          kk += 1;
        }
        cn[d] = wrap_index((long long)cc[d][k] + kk, n);
        on[d] = __float_as_int(o2);
      }
      if (ok) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          cc[d][k] = cn[d];
          oo[d][k] = on[d];
        }
      } else {
        bad = true;
      }
    }
    if (bad) set_status(status, PM_ERR_RANGE);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      reinterpret_cast<int4*>(q + d * np)[i] = make_int4(cc[d][0], cc[d][1], cc[d][2], cc[d][3]);
      reinterpret_cast<int4*>(q + (3 + d) * np)[i] = make_int4(oo[d][0], oo[d][1], oo[d][2], oo[d][3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Inspection: packed [N][N][M] -> rfftn layout [N][N][M+1].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_unpack_spec(const cx<T>* __restrict__ spec, cx<T>* __restrict__ dst, int n) {
  const int m = n / 2;
  const int64_t total = (int64_t)n * n * (m + 1);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(idx % (m + 1));
    const int64_t row = idx / (m + 1);
    if (kx > 0 && kx < m) {
      dst[idx] = spec[row * m + kx];
    } else {
      const int iz = (int)(row / n), iy = (int)(row % n);
      const int jz = (n - iz) % n, jy = (n - iy) % n;
      const cx<T> f = spec[row * m], h = spec[((int64_t)jz * n + jy) * m];
      if (kx == 0) dst[idx] = {(T)0.5 * (f.x + h.x), (T)0.5 * (f.y - h.y)};
      else dst[idx] = {(T)0.5 * (f.y + h.y), (T)-0.5 * (f.x - h.x)};
    }
  }
}

}  // namespace nupm
