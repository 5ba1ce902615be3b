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
