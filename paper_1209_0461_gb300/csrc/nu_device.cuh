// Device code of the neutrino response (Eq. P-final with Eq. deltaI-nu or
// Eq. deltaI-multipole, Sec. 4.3 (iii), App. B): the free-streaming kernel,
// the s(a) table, and the per-item bodies that the response kernels
// (nu_response.cu) and the batched kicks (batch.cu) both run.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "consts.cuh"
#include "nupm_internal.h"

namespace nupm {

// ---------------------------------------------------------------- I(x)
// Complex trigamma psi'(z), Re z > 0: recurrence psi'(z) = psi'(z+1) + 1/z^2
// up to |z| >= 9, then the Bernoulli asymptotic series.
__device__ static void trigamma(double zr, double zi, double& outr, double& outi) {
  double sr = 0.0, si = 0.0;
  while (zr * zr + zi * zi < 81.0) {
    // 1/z^2 = conj(z)^2 / |z|^4
    const double d = zr * zr + zi * zi;
    const double inv = 1.0 / (d * d);
    sr += (zr * zr - zi * zi) * inv;
    si += (-2.0 * zr * zi) * inv;
    zr += 1.0;
  }
  const double d = zr * zr + zi * zi;
  const double ir = zr / d, ii = -zi / d;            // 1/z
  const double i2r = ir * ir - ii * ii, i2i = 2.0 * ir * ii;   // 1/z^2
  // sum_k B_2k / z^{2k+1} = (1/z) sum_k B_2k (1/z^2)^k, Horner in 1/z^2
  double pr = 0.0, pi = 0.0;
  for (int k = kBernTerms - 1; k >= 0; --k) {
    const double tr = pr * i2r - pi * i2i + kBern[k];
    const double ti = pr * i2i + pi * i2r;
    pr = tr;
    pi = ti;
  }
  // psi'(z) = (1/z) (1 + y P) + y / 2 with y = 1/z^2, P = sum_k B_{2k} y^{k-1}
  const double qr = 1.0 + (pr * i2r - pi * i2i), qi = pr * i2i + pi * i2r;
  outr = sr + (ir * qr - ii * qi) + 0.5 * i2r;
  outi = si + (ir * qi + ii * qr) + 0.5 * i2i;
}

// Free-streaming kernel I(x) of the relativistic Fermi-Dirac distribution
// (Eq. I.def; App. C series):
//   x < 0.5   Taylor series in x^2 (coefficients from the Dirichlet eta function)
//   x < 24    I = Im[psi'(1 + i x/2) - psi'(1/2 + i x/2)] / (6 zeta(3) x)
//   x >= 24   asymptotic series 1/(3 zeta 3) sum_n g_n x^{-2n-2} (Genocchi g_n)
__device__ static double nu_I_exact(double x) {
  x = fabs(x);
  if (x < 0.5) {
    const double x2 = x * x;
    double s = 0.0;
    for (int j = kITaylorTerms - 1; j >= 0; --j) s = s * x2 + kITaylor[j];
    return s;
  }
  if (x < 24.0) {
    double ar, ai, br, bi;
    trigamma(1.0, 0.5 * x, ar, ai);
    trigamma(0.5, 0.5 * x, br, bi);
    return (ai - bi) / (6.0 * kZeta3 * x);
  }
  const double y = 1.0 / (x * x);
  double s = 0.0;
  for (int j = kIAsymTerms - 1; j >= 0; --j) s = s * y + kIAsym[j];
  return s * y * y / (3.0 * kZeta3);
}

// I(x) from its piecewise Chebyshev form on [kIX0, kIX0 + kISeg kIH) (the
// trigamma range of nu_I_exact; the Taylor and asymptotic branches outside it
// are cheap and stay as they are).  Piece s covers x_s = kIX0 + s kIH .. x_s + kIH
// and holds c_k, I = c_0 + sum_{k>=1} c_k T_k(t), t = 2 (x - x_s) / kIH - 1,
// evaluated by Clenshaw's recurrence.  The pieces are the Chebyshev
// interpolants at kICoef points of the first kind (k_I_table): I is analytic in
// a strip |Im x| < 1 around the real axis (poles of the trigammas at x = +-i,
// +-2i, ...), so on pieces of width 1/4 the interpolation error is ~4e-15
// relative (one twelfth of the exact evaluation's FP64 work, which dominates the
// response on a part with a low FP64 rate).
__device__ __forceinline__ double nu_I_table(double x, const double* __restrict__ c) {
  x = fabs(x);
  const double v = (x - kIX0) * (1.0 / kIH);
  if (!(v >= 0.0) || v >= (double)kISeg) return nu_I_exact(x);
  const int s = (int)v;
  const double t = 2.0 * (v - (double)s) - 1.0;
  const double* cs = c + s * kICoef;
  double b1 = 0.0, b2 = 0.0;
#pragma unroll
  for (int k = kICoef - 1; k >= 1; --k) {
    const double b0 = fma(2.0 * t, b1, cs[k] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(t, b1, cs[0] - b2);
}

// App. C fitting formula (Eq. fit).
__device__ static double nu_I_fit(double x) {
  x = fabs(x);
  const double x2 = x * x;
  const double num = 1.0 + 0.0168 * x2 + 0.0407 * x2 * x2;
  const double den = 1.0 + 2.1734 * x2 + 1.6787 * pow(x, 4.1811) + 0.1467 * x2 * x2 * x2 * x2;
  return num / den;
}

// s(u) - s(u_i) from the cubic-Hermite table (values and ds/du at each node).
__device__ __forceinline__ double s_table(const NuArgs& A, double u) {
  double t = (u - A.stab_u0) * A.stab_inv_h;
  int i = (int)floor(t);
  if (i < 0) i = 0;
  if (i > A.n_stab - 2) i = A.n_stab - 2;
  t -= (double)i;
  const double s0 = A.stab[2 * i], d0 = A.stab[2 * i + 1] * A.stab_h;
  const double s1 = A.stab[2 * i + 2], d1 = A.stab[2 * i + 3] * A.stab_h;
  const double t2 = t * t, t3 = t2 * t;
  return (2 * t3 - 3 * t2 + 1) * s0 + (t3 - 2 * t2 + t) * d0 + (-2 * t3 + 3 * t2) * s1 + (t3 - t2) * d1;
}

struct Panel {
  double lo, hi;
  int seg;   // history interval: -1 before node 0, j in [0, n-1) between nodes, n-1 the last
};

// One warp per (bin, species, chunk of 32 panels): partial IC, J_hist, W_cur.
// The l = 1 term of Eq. deltaI-multipole for the initial moments of Sec. 4.1
// (delta f_1 = f_0' m a_i theta / k), K(y) = -(1/y) int u^2 f'(u) j_1(u y) du /
// ((3/2) zeta(3)), f = 1 / (e^u + 1), by Gauss-Legendre panels on [0, 50] of
// width min(1/2, 3/(2 y)) (a quarter period of j_1 at most), the panels dealt
// to the lanes of a warp and summed in a fixed order.  Every lane returns K.
// Beyond y = kMultipoleYMax (where K < 1e-10) the integrated-by-parts value
// I(y) stands in.
constexpr double kMultipoleYMax = 256.0;
__device__ static double sph_j1(double z) {
  if (z < 1e-2) {
    const double z2 = z * z;
    return z * (1.0 / 3.0 - z2 * (1.0 / 30.0 - z2 / 840.0));
  }
  return (sin(z) / z - cos(z)) / z;
}
__device__ static double nu_K_warp(double y, const NuArgs& A, int lane) {
  if (y <= 0.0) return 1.0;
  const double U = 50.0;
  const double hmax = fmin(0.5, 1.5 / y);
  const int np = (int)ceil(U / hmax);
  const double h = U / np;
  double acc = 0.0;
  for (int p = lane; p < np; p += 32) {
    const double lo = p * h;
    double ps = 0.0;
    for (int q = 0; q < A.quad; ++q) {
      const double u = lo + 0.5 * h * (A.gl[q] + 1.0);
      const double e = exp(-u);
      const double fp = -e / ((1.0 + e) * (1.0 + e));
      ps += A.gl[kMaxQuad + q] * u * u * fp * sph_j1(u * y);
    }
    acc += 0.5 * h * ps;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return -acc / (y * 1.5 * kRelZeta3);
}

// Body: the panel chunk `item` (< nk ns kNuChunks) of (bin, species), one warp
// (warp w of the CTA's four uses panel scratch w).
__device__ __forceinline__ void nu_panels_item(const NuArgs& A, int item) {
  __shared__ Panel panels[4][kMaxPanels];
  __shared__ int npan[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (item >= A.nk * A.ns * kNuChunks) return;
  const int chunk = item % kNuChunks;
  if (chunk >= A.nchunks) return;        // unused chunk: nothing written, nothing read
  const int bs = item / kNuChunks;
  const int b = bs % A.nk, s = bs / A.nk;
  double* out = A.parts + (int64_t)item * 3;
  const double cnt = A.bins[b];
  if (cnt <= 0.0) {
    if (lane == 0) out[0] = out[1] = out[2] = 0.0;
    return;
  }
  const double kb = A.bins[A.nk + b] / cnt;
  const double s_end = s_table(A, A.ue);
  const double kappa = kb * A.kappa_scale[s];
  const double Ha = A.rel ? sqrt(rel_e2(A.a, A.bg)) : sqrt(A.omega_m * exp(-3.0 * A.ue) + A.omega_l);
  const double ell = (kappa > 0.0) ? A.a * A.a * Ha / kappa : 1e300;
  const int n = A.n_hist;
  Panel* P = panels[warp];
  if (lane == 0) {
    // merge (descending from ln a): history nodes inside (u_i, u_e) and graded points
    int np = 0;
    double cur = A.ue;
    int j = n - 1;                       // next history node below cur
    while (j >= 0 && !(A.hist_u[j] < A.ue)) --j;
    int mexp = -2;
    double gpt = A.ue - ell * ldexp(1.0, mexp);
    while (cur > A.ui && np < kMaxPanels) {
      const double hn = (j >= 0 && A.hist_u[j] > A.ui) ? A.hist_u[j] : A.ui;
      const double gp = (gpt > A.ui) ? gpt : A.ui;
      const double nxt = hn > gp ? hn : gp;
      // the interval index of (nxt, cur): the history node at or below nxt
      P[np].lo = nxt;
      P[np].hi = cur;
      P[np].seg = j;                     // cur lies above node j (or below node 0 if j < 0)
      ++np;
      if (nxt == hn && j >= 0 && A.hist_u[j] > A.ui) --j;
      if (nxt == gp && gpt > A.ui) {
        ++mexp;
        gpt = A.ue - ell * ldexp(1.0, mexp);
      }
      while (gpt >= nxt && gpt > A.ui) {   // skip graded points at or above the new cur
        ++mexp;
        gpt = A.ue - ell * ldexp(1.0, mexp);
      }
      cur = nxt;
    }
    npan[warp] = np;
  }
  __syncwarp();
  const int np = npan[warp];
  const int Q = A.quad;
  double jh = 0.0, wc = 0.0;
  for (int pi = chunk * 32 + lane; pi < np; pi += 32 * A.nchunks) {
    const Panel pn = P[pi];
    if (!(pn.hi > pn.lo)) continue;
    const double half = 0.5 * (pn.hi - pn.lo);
    // P_M^{1/2} on this panel: h(u) = h0 + (h1 - h0) (u - u0) / (u1 - u0) (history part)
    // plus the current-node hat on the last interval
    const int seg = pn.seg;
    double u0 = 0.0, u1 = 1.0, h0 = 0.0, h1 = 0.0;
    bool last = false, before = false;
    if (n == 0) {
      last = true;                      // h == h_cur on [u_i, u_e]
    } else if (seg < 0) {
      before = true;                    // constant h_0 before the first node
      h0 = A.hist[b];
    } else if (seg == n - 1) {
      last = true;
      u0 = A.hist_u[n - 1];
      u1 = A.ue;
      h0 = A.hist[(int64_t)(n - 1) * A.nk + b];
    } else {
      u0 = A.hist_u[seg];
      u1 = A.hist_u[seg + 1];
      h0 = A.hist[(int64_t)seg * A.nk + b];
      h1 = A.hist[(int64_t)(seg + 1) * A.nk + b];
    }
    for (int q = 0; q < Q; ++q) {
      const double u = pn.lo + half * (A.gl[q] + 1.0);
      const double wq = half * A.gl[kMaxQuad + q];
      const double ap = exp(u);
      const double Hp = A.rel ? sqrt(rel_e2(ap, A.bg)) : sqrt(A.omega_m / (ap * ap * ap) + A.omega_l);
      const double ds = s_end - s_table(A, u);
      const double x = kappa * ds;
      const double I = A.use_fit ? nu_I_fit(x) : nu_I_table(x, A.icheb);
      const double base = wq * I * ds / (ap * Hp);
      if (n == 0) {
        wc += base;
      } else if (before) {
        jh += base * h0;
      } else if (last) {
        const double tau = (u - u0) / (u1 - u0);
        jh += base * h0 * (1.0 - tau);
        wc += base * tau;
      } else {
        const double tau = (u - u0) / (u1 - u0);
        jh += base * (h0 + (h1 - h0) * tau);
      }
    }
  }
  // fixed-order warp reduction
  for (int off = 16; off > 0; off >>= 1) {
    jh += __shfl_down_sync(0xffffffffu, jh, off);
    wc += __shfl_down_sync(0xffffffffu, wc, off);
  }
  // l = 1 term of Eq. deltaI-multipole by its own momentum integral (the warp's lanes)
  const double xi = kappa * s_end;
  const double Kl1 = (A.ic_multipole && chunk == 0 && xi < kMultipoleYMax) ? nu_K_warp(xi, A, lane) : 0.0;
  if (lane == 0) {
    double ic = 0.0;
    if (chunk == 0) {
      const double Ii = A.use_fit ? nu_I_fit(xi) : nu_I_table(xi, A.icheb);
      const double P = A.pnu_init[(int64_t)s * A.nk + b], th = A.theta_init[(int64_t)s * A.nk + b];
      if (A.ic_multipole)   // Eq. deltaI-multipole with the l = 0 and l = 1 moments of Sec. 4.1
        ic = P * (Ii - s_end * A.a_init * th * (xi < kMultipoleYMax ? Kl1 : Ii));
      else                  // Eq. deltaI-nu
        ic = Ii * P * (1.0 - s_end * A.a_init * th);
    }
    const double c = 1.5 * A.omega_m;
    out[0] = ic;
    out[1] = c * jh;
    out[2] = c * wc;
  }
}

// Species sum, implicit iterations, ratio (one thread per bin).
__device__ __forceinline__ void nu_finish_bin(const NuArgs& A, int b) {
  if (b >= A.nk) return;
  const double cnt = A.bins[b];
  double R = 0.0, pnu = 0.0, pm = 0.0;
  if (cnt > 0.0) {
    const double L3 = A.box * A.box * A.box;
    const double n3 = (double)A.ngrid * A.ngrid * A.ngrid;
    const double pcdm = sqrt(A.bins[2 * A.nk + b] / cnt * L3 / (n3 * n3));
    double ic = 0.0, jh = 0.0, wc = 0.0, guess = 0.0;
    for (int s = 0; s < A.ns; ++s) {
      double qi = 0.0, qj = 0.0, qw = 0.0;
      for (int ch = 0; ch < A.nchunks; ++ch) {   // fixed chunk order
        const double* q = A.parts + (((int64_t)s * A.nk + b) * kNuChunks + ch) * 3;
        qi += q[0];
        qj += q[1];
        qw += q[2];
      }
      ic += A.w_species[s] * qi;
      jh += A.w_species[s] * qj;
      wc += A.w_species[s] * qw;
      guess += A.w_species[s] * A.pnu_init[(int64_t)s * A.nk + b];
    }
    if (A.prev) guess = A.prev[b];
    pnu = guess;
    for (int it = 0; it < A.iters; ++it)
      pnu = ic + jh + ((1.0 - A.f_nu) * pcdm + A.f_nu * pnu) * wc;
    R = pcdm > 0.0 ? pnu / pcdm : 0.0;
    pm = (1.0 - A.f_nu) * pcdm + A.f_nu * pnu;
  }
  A.R[b] = R;
  A.pnu[b] = pnu;
  A.pm[b] = pm;
  if (A.R_user) A.R_user[b] = R;
  if (A.pnu_user) A.pnu_user[b] = pnu;
  if (A.pm_user) A.pm_user[b] = pm;
}


// Compacted (ln k_b, R_b) of the non-empty bins, in bin order, for the Green
// and fac tables: rlist[0..c) = ln k_b, rlist[nk..nk+c) = R_b, rlist[2 nk] = c.
// One block of nk <= 1024 threads.
__device__ __forceinline__ void nu_rlist_block(const double* __restrict__ bins, const double* __restrict__ R, int nk,
                                               double* __restrict__ rlist) {
  __shared__ int warp_cnt[32];
  const int b = threadIdx.x, lane = b & 31, warp = b >> 5;
  const bool ne = b < nk && bins[b] > 0.0;
  const unsigned m = __ballot_sync(0xffffffffu, ne);
  if (lane == 0) warp_cnt[warp] = __popc(m);
  __syncthreads();
  int base = 0;
  for (int w = 0; w < warp; ++w) base += warp_cnt[w];
  const int pos = base + __popc(m & ((1u << lane) - 1));
  if (ne) {
    rlist[pos] = log(bins[nk + b] / bins[b]);
    rlist[nk + pos] = R[b];
  }
  if (b == blockDim.x - 1) rlist[2 * nk] = (double)(base + __popc(m));
}


// fac table for the FP32 Green function: the same ln-k interpolation of R as
// k_green_table, sampled on a uniform grid of u = ln(k / kf).
// Body: table entries j0, j0 + step, ... (the non-empty bins staged in the
// CTA's dynamic shared memory, 2 nk doubles).
__device__ __forceinline__ void fac_table_entries(float* __restrict__ fac, double umax, double kf, double f_nu,
                                                  const double* __restrict__ rlist, int nk, int j0, int step) {
  extern __shared__ double sh[];
  double* lk = sh;
  double* rv = sh + nk;
  const int cnum = (int)rlist[2 * nk];
  for (int i = threadIdx.x; i < cnum; i += blockDim.x) {
    lk[i] = rlist[i];
    rv[i] = rlist[nk + i];
  }
  __syncthreads();
  const double lkf = log(kf);
  for (int j = j0; j < kFacTable; j += step) {
    double r = 0.0;
    if (f_nu > 0.0 && cnum > 0) {
      const double l = lkf + umax * (double)j / (double)(kFacTable - 1);
      if (l <= lk[0]) {
        r = rv[0];
      } else if (l >= lk[cnum - 1]) {
        r = rv[cnum - 1];
      } else {
        int lo = 0, hi = cnum - 1;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (lk[mid] <= l) lo = mid; else hi = mid;
        }
        r = rv[lo] + (rv[hi] - rv[lo]) * (l - lk[lo]) / (lk[hi] - lk[lo]);
      }
    }
    fac[j] = (float)((1.0 - f_nu) + f_nu * r);
  }
}

// Outputs i0 .. i0 + 31 of out[i] = sum_blk partials[blk][i], blk < nblk: warp w
// adds rows w, w + kReduceWarps, ... for lane i0 + lane (coalesced), then one
// warp adds the kReduceWarps warp sums in warp order -- a fixed order, so the
// result is the same at every run.  blockDim = kReduceWarps * 32.
constexpr int kReduceWarps = 32;
__device__ __forceinline__ void bin_reduce_group(const double* __restrict__ partials, int nblk, int len,
                                                 double* __restrict__ out, int i0) {
  __shared__ double red[kReduceWarps][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = i0 + lane;
  double acc = 0.0;
  if (i < len)
    for (int b = warp; b < nblk; b += kReduceWarps) acc += partials[(int64_t)b * len + i];
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < kReduceWarps; ++w) s += red[w][lane];
    if (i < len) out[i] = s;
  }
}

}  // namespace nupm
