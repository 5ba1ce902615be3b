// Neutrino linear response per |k| bin, FP64 on the GPU (Eq. P-final with the
// initial-condition term Eq. deltaI-nu, the implicit solve of Sec. 4.3 (iii)
// and App. B), and the Green table of the total-matter force (Eq. phases,
// Sec. 4.3 (iv), Eq. Poisson).
//
// For bin b and species s (kappa = k_b c/H0 T_nu0 / m_s, x = kappa (s - s')):
//   IC_s  = I(kappa s(a)) P_nu,i^{1/2} (1 - s(a) a_i [theta/delta]_i)
//   J_s   = 3/2 Omega_M int_{ln a_i}^{ln a} I(x) (s - s') P_M^{1/2}(a') / (a' H(a')) dln a'
// P_M^{1/2} is linear in ln a' between stored nodes, constant before the
// first, and its last node is the current value
//   h_cur = (1 - f_nu) P_cdm^{1/2}(a) + f_nu P_nu^{1/2}(guess).
// J is linear in h_cur: J = J_hist + h_cur W_cur, so every iteration of the
// implicit equation is free once (IC, J_hist, W_cur) are known.
//
// Quadrature: Gauss-Legendre panels in ln a'.  Break points are the stored
// nodes (kinks of the interpolant) and the graded points ln a - l 2^m,
// m = -2, -1, ..., with l = a^2 H(a) / kappa the ln-a width over which
// kappa (s - s') reaches one: the integrand is smooth on each panel.
#include <cuda_runtime.h>
#include <math.h>

#include "consts.cuh"
#include "nu_device.cuh"
#include "nupm_internal.h"

namespace nupm {

__global__ void k_nu_panels(NuArgs A) { nu_panels_item(A, blockIdx.x * 4 + (threadIdx.x >> 5)); }

__global__ void k_nu_finish(NuArgs A) { nu_finish_bin(A, blockIdx.x * blockDim.x + threadIdx.x); }

// Fixed-order sum of the per-CTA bin partials: out[i] = sum_blk partials[blk][i]
// (bin_reduce_group: a CTA of kReduceWarps warps, 32 outputs).
__global__ void __launch_bounds__(kReduceWarps * 32) k_bin_reduce(const double* __restrict__ partials, int nblk,
                                                                 int len, double* __restrict__ out) {
  bin_reduce_group(partials, nblk, len, out, blockIdx.x * 32);
}

__global__ void k_nu_rlist(const double* __restrict__ bins, const double* __restrict__ R, int nk,
                           double* __restrict__ rlist) {
  nu_rlist_block(bins, R, nk, rlist);
}

// Chebyshev pieces of I(x) (nu_I_table): block s evaluates the exact I at the
// kICoef points x_s + kIH (1 + cos(pi (j + 1/2) / kICoef)) / 2 and transforms
// them to c_k = (2 / kICoef) sum_j I_j cos(pi k (j + 1/2) / kICoef), c_0 halved.
__global__ void k_I_table(double* __restrict__ coef) {
  __shared__ double f[kICoef];
  const int s = blockIdx.x, j = threadIdx.x;
  const double t = cospi((j + 0.5) / kICoef);
  f[j] = nu_I_exact(kIX0 + kIH * s + 0.5 * kIH * (t + 1.0));
  __syncthreads();
  double c = 0.0;
  for (int i = 0; i < kICoef; ++i) c += f[i] * cospi((double)j * (i + 0.5) / kICoef);
  c *= 2.0 / kICoef;
  coef[s * kICoef + j] = j == 0 ? 0.5 * c : c;
}

void launch_I_table(double* coef, cudaStream_t s) { k_I_table<<<kISeg, kICoef, 0, s>>>(coef); }

void launch_nu_panels(const NuArgs& a, cudaStream_t s) {
  const int items = a.nk * a.ns * kNuChunks;
  if (items > 0) k_nu_panels<<<(items + 3) / 4, 128, 0, s>>>(a);
}

void launch_nu_finish(const NuArgs& a, cudaStream_t s) {
  k_nu_finish<<<(a.nk + 127) / 128, 128, 0, s>>>(a);
  k_nu_rlist<<<1, ((a.nk + 31) / 32) * 32, 0, s>>>(a.bins, a.R, a.nk, a.rlist);
}

void launch_nu_response(const NuArgs& a, cudaStream_t s) {
  launch_nu_panels(a, s);
  launch_nu_finish(a, s);
}

// ---------------------------------------------------------------- surrogate
// Features of bin b for the learned response (FP64, one thread per bin):
//   (ln k_b, ln a, M_nu, Omega_nu, c_0 .. c_7), c_j the Chebyshev coefficients
// on 8 points of g(u) = ln(P_M^{1/2}(u) / P_cdm^{1/2}(a)), u = ln a' in
// [ln a_i, ln a]; P_M^{1/2} linear in u between the nodes (hist_u[j], hist[j][b])
// closed by (ln a, P_cdm^{1/2}), constant before the first node.
__global__ void k_nu_features(NuArgs A, double m_nu, double omega_nu, float* __restrict__ X) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.nk) return;
  float* row = X + (int64_t)b * 12;
  const double cnt = A.bins[b];
  if (!(cnt > 0.0)) {
    for (int i = 0; i < 12; ++i) row[i] = 0.0f;
    return;
  }
  const double L3 = A.box * A.box * A.box;
  const double n3 = (double)A.ngrid * A.ngrid * A.ngrid;
  const double pcdm = sqrt(A.bins[2 * A.nk + b] / cnt * L3 / (n3 * n3));
  const double kb = A.bins[A.nk + b] / cnt;
  double g[8];
  for (int m = 0; m < 8; ++m) {
    const double t = cospi((m + 0.5) / 8.0);
    const double u = A.ui + 0.5 * (t + 1.0) * (A.ue - A.ui);
    double h = pcdm;
    if (A.n_hist > 0) {
      if (u <= A.hist_u[0]) {
        h = A.hist[b];
      } else {
        int j = 0;
        while (j + 1 < A.n_hist && A.hist_u[j + 1] < u) ++j;
        const double u0 = A.hist_u[j], h0 = A.hist[(int64_t)j * A.nk + b];
        const double u1 = j + 1 < A.n_hist ? A.hist_u[j + 1] : A.ue;
        const double h1 = j + 1 < A.n_hist ? A.hist[(int64_t)(j + 1) * A.nk + b] : pcdm;
        h = h0 + (h1 - h0) * (u - u0) / (u1 - u0);
      }
    }
    g[m] = (h > 0.0 && pcdm > 0.0) ? log(h / pcdm) : 0.0;
  }
  row[0] = (float)log(kb);
  row[1] = (float)A.ue;
  row[2] = (float)m_nu;
  row[3] = (float)omega_nu;
  for (int jc = 0; jc < 8; ++jc) {
    double c = 0.0;
    for (int m = 0; m < 8; ++m) c += g[m] * cospi(jc * (m + 0.5) / 8.0);
    row[4 + jc] = (float)(0.25 * c);
  }
}

// R_b = exp(ln R_b) from the surrogate, then P_nu^{1/2} and P_M^{1/2} as the
// exact finish does (empty bins: 0).
__global__ void k_nu_from_lnR(NuArgs A, const float* __restrict__ lnR) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.nk) return;
  const double cnt = A.bins[b];
  double R = 0.0, pnu = 0.0, pm = 0.0;
  if (cnt > 0.0) {
    const double L3 = A.box * A.box * A.box;
    const double n3 = (double)A.ngrid * A.ngrid * A.ngrid;
    const double pcdm = sqrt(A.bins[2 * A.nk + b] / cnt * L3 / (n3 * n3));
    R = exp((double)lnR[b]);
    pnu = R * pcdm;
    pm = (1.0 - A.f_nu) * pcdm + A.f_nu * pnu;
  }
  A.R[b] = R;
  A.pnu[b] = pnu;
  A.pm[b] = pm;
  if (A.R_user) A.R_user[b] = R;
  if (A.pnu_user) A.pnu_user[b] = pnu;
  if (A.pm_user) A.pm_user[b] = pm;
}

void launch_nu_features(const NuArgs& a, double m_nu, double omega_nu, float* X, cudaStream_t s) {
  k_nu_features<<<(a.nk + 127) / 128, 128, 0, s>>>(a, m_nu, omega_nu, X);
}

void launch_nu_from_lnR(const NuArgs& a, const float* lnR, cudaStream_t s) {
  k_nu_from_lnR<<<(a.nk + 127) / 128, 128, 0, s>>>(a, lnR);
  k_nu_rlist<<<1, ((a.nk + 31) / 32) * 32, 0, s>>>(a.bins, a.R, a.nk, a.rlist);
}

// ---------------------------------------------------------------- Green table
// G(n^2) = coeff [(1 - f) + f R(k)] / n^2, k = kf sqrt(n^2); R linear in ln k
// between non-empty bins (k_b = ksum/count), constant beyond the end bins.
template <typename T>
__global__ void k_green_table(T* __restrict__ gtab, long long n2max, double kf, double coeff,
                              double f_nu, const double* __restrict__ rlist, int nk) {
  extern __shared__ double sh[];
  double* lk = sh;          // ln k of non-empty bins
  double* rv = sh + nk;     // their R
  const int cnum = (int)rlist[2 * nk];
  for (int i = threadIdx.x; i < cnum; i += blockDim.x) {
    lk[i] = rlist[i];
    rv[i] = rlist[nk + i];
  }
  __syncthreads();
  for (long long n2 = (long long)blockIdx.x * blockDim.x + threadIdx.x; n2 <= n2max;
       n2 += (long long)gridDim.x * blockDim.x) {
    if (n2 == 0) {
      gtab[0] = (T)0;
      continue;
    }
    double r = 0.0;
    if (f_nu > 0.0 && cnum > 0) {
      const double l = log(kf * sqrt((double)n2));
      if (l <= lk[0]) {
        r = rv[0];
      } else if (l >= lk[cnum - 1]) {
        r = rv[cnum - 1];
      } else {
        int lo = 0, hi = cnum - 1;   // lk[lo] <= l < lk[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (lk[mid] <= l) lo = mid; else hi = mid;
        }
        r = rv[lo] + (rv[hi] - rv[lo]) * (l - lk[lo]) / (lk[hi] - lk[lo]);
      }
    }
    gtab[n2] = (T)(coeff * ((1.0 - f_nu) + f_nu * r) / (double)n2);
  }
}

__global__ void k_fac_table(float* __restrict__ fac, double umax, double kf, double f_nu,
                            const double* __restrict__ rlist, int nk) {
  fac_table_entries(fac, umax, kf, f_nu, rlist, nk, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

void launch_fac_table(float* fac, double umax, double kf, double f_nu, const double* rlist, int nk,
                      cudaStream_t s) {
  k_fac_table<<<(kFacTable + 255) / 256, 256, 2 * (size_t)nk * sizeof(double), s>>>(fac, umax, kf, f_nu, rlist, nk);
}

void launch_green_table(bool fp64, void* gtab, long long n2max, double kf, double coeff,
                        double f_nu, const double* rlist, int nk, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (n2max + 1 + threads - 1) / threads;
  if (blocks > 1216) blocks = 1216;
  const size_t sh = 2 * (size_t)nk * sizeof(double);
  if (fp64)
    k_green_table<double><<<(int)blocks, threads, sh, s>>>((double*)gtab, n2max, kf, coeff, f_nu, rlist, nk);
  else
    k_green_table<float><<<(int)blocks, threads, sh, s>>>((float*)gtab, n2max, kf, coeff, f_nu, rlist, nk);
}

}  // namespace nupm
