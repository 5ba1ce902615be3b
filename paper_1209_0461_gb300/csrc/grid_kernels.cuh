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
            if (wt) atomicAdd(grid + rowi + xs[dx], wt);
          }
        }
    }
  }
}

// Signed frequency of index i on an n-point axis.
__device__ __forceinline__ int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// ---------------------------------------------------------------------------
// a3: binned power of the packed spectrum, deterministic.  One warp per row
// (z, y); lanes take consecutive x2.  Along a row n^2 = kz^2 + ky^2 + x2^2 grows
// with x2, so the bins of a 32-lane chunk are contiguous lane segments: a
// segmented shuffle scan sums each segment and its last lane adds the sum to
// the warp's private accumulator (one writer per bin, no atomics).  Warps and
// CTAs are then summed in a fixed order (k_bin_reduce).  The bin of each n^2
// comes from a lookup table (bin_of[n2], -1 outside the bins).
//   LATTICE = true : accumulate the mode count sum w and sum w |k| (depends on
//                    the lattice only; run once per context)
//   LATTICE = false: accumulate sum w |delta_k|^2; per-mode arithmetic in the
//                    grid precision T, one FP64 add per segment
// The packed slot x2 = 0 is unpacked with the row at (-z, -y):
//   A = (F(k) + conj F(-k)) / 2   (kx = 0),  B = (F(k) - conj F(-k)) / (2i)  (kx = N/2).
// Shared memory: [kBinWarps][NV][nk] doubles (NV = 2 lattice sums or 1).
// ---------------------------------------------------------------------------
constexpr int kBinWarps = 4;
constexpr int kBinBatch = 8;   // chunks loaded per batch (bytes in flight)

template <typename T, bool LATTICE>
__global__ void __launch_bounds__(kBinWarps * 32)
k_bin_power(const cx<T>* __restrict__ spec, int n, int nk, const short* __restrict__ bin_of,
            double kf, double* __restrict__ partials) {
  constexpr int NV = LATTICE ? 2 : 1;
  using A = typename std::conditional<LATTICE, double, T>::type;   // scan type
  // FP32 power: per-row sums in FP32 (at most M modes a bin), added to the
  // warp's FP64 sums once per row (GB300's FP64 pipe is narrow)
  constexpr bool ROWF = !LATTICE && sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* all = reinterpret_cast<double*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = all + warp * NV * nk;
  float* racc = reinterpret_cast<float*>(all + kBinWarps * NV * nk) + warp * nk;
  for (int i = threadIdx.x; i < kBinWarps * NV * nk; i += blockDim.x) all[i] = 0.0;
  if constexpr (ROWF)
    for (int i = threadIdx.x; i < kBinWarps * nk; i += blockDim.x) racc[i - warp * nk] = 0.0f;
  __syncthreads();
  const unsigned full = 0xffffffffu;
  const int m = n / 2;
  const int rows = n * n;
  for (int row = blockIdx.x * kBinWarps + warp; row < rows; row += gridDim.x * kBinWarps) {
    const int iz = row / n, iy = row - (row / n) * n;
    const int kz = signed_freq(iz, n), ky = signed_freq(iy, n);
    const int base2 = kz * kz + ky * ky;
    const cx<T>* r = spec + (int64_t)row * m;
    for (int x0 = 0; x0 < m; x0 += 32 * kBinBatch) {
      cx<T> f[kBinBatch];
      if constexpr (!LATTICE) {
#pragma unroll
        for (int j = 0; j < kBinBatch; ++j) {
          const int x2 = x0 + 32 * j + lane;
          f[j] = x2 < m ? r[x2] : cx<T>{(T)0, (T)0};
        }
      }
#pragma unroll
      for (int j = 0; j < kBinBatch; ++j) {
        const int x2 = x0 + 32 * j + lane;
        if (x0 + 32 * j >= m) break;                     // warp-uniform
        A v0 = 0, v1 = 0;
        int b = -1;
        if (x2 > 0 && x2 < m) {
          const int n2 = base2 + x2 * x2;
          b = bin_of[n2];
          if constexpr (LATTICE) {
            v0 = 2.0;
            v1 = 2.0 * kf * sqrt((double)n2);
          } else {
            v0 = (T)2 * (f[j].x * f[j].x + f[j].y * f[j].y);
          }
        } else if (x2 == 0) {
          const int n2b = base2 + m * m;                 // kx = N/2 mode: added directly
          const int bb = bin_of[n2b];
          b = bin_of[base2];                             // kx = 0 mode joins the scan
          if constexpr (LATTICE) {
            v0 = 1.0;
            v1 = kf * sqrt((double)base2);
            if (bb >= 0) {
              acc[bb] += 1.0;
              acc[nk + bb] += kf * sqrt((double)n2b);
            }
          } else {
            const int jz = partner_index(iz, n), jy = partner_index(iy, n);
            const cx<T> g = spec[((int64_t)jz * n + jy) * m];
            const T ax = (T)0.5 * (f[j].x + g.x), ay = (T)0.5 * (f[j].y - g.y);
            const T bx = (T)0.5 * (f[j].y + g.y), by = (T)-0.5 * (f[j].x - g.x);
            v0 = ax * ax + ay * ay;
            if (bb >= 0) {
              if constexpr (ROWF) racc[bb] += (float)(bx * bx + by * by);
              else acc[bb] += (double)(bx * bx + by * by);
            }
          }
        }
        if (b < 0) v0 = v1 = 0;
        __syncwarp();
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const A p0 = __shfl_up_sync(full, v0, off);
          A p1 = 0;
          if constexpr (LATTICE) p1 = __shfl_up_sync(full, v1, off);
          const int b2 = __shfl_up_sync(full, b, off);
          if (lane >= off && b2 == b) {
            v0 += p0;
            if constexpr (LATTICE) v1 += p1;
          }
        }
        const int bn = __shfl_down_sync(full, b, 1);
        if (b >= 0 && (lane == 31 || bn != b)) {
          if constexpr (ROWF) {
            racc[b] += (float)v0;
          } else {
            acc[b] += (double)v0;
            if constexpr (LATTICE) acc[nk + b] += (double)v1;
          }
        }
        __syncwarp();
      }
    }
    if constexpr (ROWF) {
      // the row's modes have n^2 in [base2, base2 + m^2]: bins b_lo .. b_hi
      // (bin_of is non-decreasing where it is >= 0; -1 ends fall back to all bins)
      int b_lo = bin_of[base2 == 0 ? 1 : base2], b_hi = bin_of[base2 + m * m];
      if (b_lo < 0) b_lo = 0;
      if (b_hi < 0) b_hi = nk - 1;
      for (int b = b_lo + lane; b <= b_hi; b += 32) {
        acc[b] += (double)racc[b];
        racc[b] = 0.0f;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV * nk; i += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int wi = 0; wi < kBinWarps; ++wi) sum += all[wi * NV * nk + i];
    partials[(int64_t)blockIdx.x * NV * nk + i] = sum;
  }
}

// ---------------------------------------------------------------------------
// a5 on the packed column x2 = 0: its slot holds A + i B, the kx = 0 and
// kx = N/2 plane spectra, whose Green factors differ.  Unpack with the
// partner at (-ky, -kz), multiply each by its G(n^2) (and deconvolution), and
// repack P = G_A A + i G_B B into plane0[ky][kz] for k_fft_z_inv_green.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_green_plane0(const cx<T>* __restrict__ spec, cx<T>* __restrict__ plane0, int n,
                               const T* __restrict__ gtab, const T* __restrict__ wtab) {
  const int m = n / 2;
  const int total = n * n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int iy = idx / n, iz = idx - (idx / n) * n;    // plane0 layout [ky][kz]
    const int ky = signed_freq(iy, n), kz = signed_freq(iz, n);
    const int jy = partner_index(iy, n), jz = partner_index(iz, n);
    const cx<T> f = spec[((int64_t)iz * n + iy) * m];
    const cx<T> h = spec[((int64_t)jz * n + jy) * m];
    const cx<T> A = {(T)0.5 * (f.x + h.x), (T)0.5 * (f.y - h.y)};
    const cx<T> B = {(T)0.5 * (f.y + h.y), (T)-0.5 * (f.x - h.x)};
    const int n2a = ky * ky + kz * kz;
    T ga = gtab[n2a], gb = gtab[n2a + m * m];
    if (wtab) {
      const T wyz = wtab[iy] * wtab[iz];
      ga *= wtab[0] * wyz;
      gb *= wtab[m] * wyz;
    }
    plane0[idx] = {ga * A.x - gb * B.y, ga * A.y + gb * B.x};   // G_A A + i G_B B
  }
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

template <typename T>
__global__ void __launch_bounds__(128)
k_interp_kick_fd(const void* __restrict__ pos, int64_t np, int n, double delta, const T* __restrict__ phi,
                 T* __restrict__ vel, T kick, T* __restrict__ acc_out, int* status) {
  const T scale = (T)(-1.0 / (12.0 * delta));   // acc = -S phi
  const T inv = (T)1.0 / (T)kWeightOne;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // the next particle's position words are fetched while this one's
  // potential values are in flight (one memory round trip per particle)
  typename Quant<T>::Raw next;
  if (p < np) next = Quant<T>::load(pos, np, p);
  for (; p < np; p += stride) {
    const typename Quant<T>::Raw raw = next;
    if (p + stride < np) next = Quant<T>::load(pos, np, p + stride);
    const T u0 = vel[p], u1 = vel[np + p], u2 = vel[2 * np + p];
    int c[3], w[3];
    if (!Quant<T>::get(raw, n, delta, c, w, status)) continue;
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
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const T* r = phi + row(ys[2 + dy], zs[2 + dz]);
#pragma unroll
        for (int j = 0; j < 6; ++j) px[dz][dy][j] = r[xs[j]];
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
    T a[3] = {(T)0, (T)0, (T)0};
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
    const T u[3] = {u0, u1, u2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T ad = a[d] * scale;
      vel[d * np + p] = u[d] + ad * kick;
      if (acc_out) acc_out[d * np + p] = ad;
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
