// Host side of the C ABI declared in include/nupm.h: argument checks,
// context and device memory, FP64 host tables, and the launch sequence of
// one kick (Sec. 4.3 steps (ii)-(iv) of the paper).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "nupm_internal.h"

using namespace nupm;

struct pm_ctx {
  pm_params p{};
  cudaStream_t stream = nullptr;
  bool fp64 = true;
  int n = 0, m = 0, nk = 0, ns = 0, quad = 8, iters = 1;
  int64_t np = 0;
  double box = 0, delta = 0, kf = 0, omega_m = 0, omega_l = 0, omega_nu = 0, f_nu = 0, a_init = 0;
  double mass[3] = {0, 0, 0}, wsp[3] = {0, 0, 0};
  int64_t n2max = 0, field_elems = 0;
  size_t cplx = 0;            // bytes of one complex element
  int nblk_bins = 0;
  // device memory
  void* spec = nullptr;       // packed spectrum
  void* g = nullptr;          // 3 packed fields (deposit grid aliases the first two)
  void* tw_n = nullptr;
  void* tw_m = nullptr;
  int* d_thr = nullptr;        // bin thresholds T_0..T_nk (int32)
  float bin_inv_lr = 0;        // nk / ln r^2: the bin of n^2 is floor(nk ln n^2 / ln r^2)
  double* d_partials = nullptr;
  double* d_bins = nullptr;   // [3][nk]
  double* d_pi = nullptr;     // [ns][nk]
  double* d_ti = nullptr;
  double* d_stab = nullptr;
  int n_stab = 0;
  double stab_u0 = 0, stab_h = 0, stab_umax = 0;
  double* d_hist_u = nullptr;
  double* d_gl = nullptr;
  double* d_parts = nullptr;  // [ns][nk][3]
  double* d_R = nullptr;
  double* d_pnu = nullptr;
  double* d_pm = nullptr;
  double* d_rlist = nullptr;  // [2 nk + 1] compacted non-empty (ln k_b, R_b)
  void* d_gtab = nullptr;
  void* d_dtab = nullptr;
  void* d_wtab = nullptr;
  void* d_plane0 = nullptr;   // [N][N] complex, Green-multiplied packed column
  float* d_fac = nullptr;     // fac table of the FP32 Green function
  int* d_rowc = nullptr;      // particle row sort: counts, starts, cursors, scan totals, perm
  int* d_rows = nullptr;
  int* d_rowcur = nullptr;
  int* d_scantot = nullptr;
  int* d_perm = nullptr;
  unsigned long long* d_rec = nullptr;
  // TMA tensor maps of the column passes (spectrum along y / z, fields along y)
  bool tma = false;
  alignas(64) CUtensorMap tm_spec_y, tm_spec_z, tm_g_y;
  // spectrum along z with 128-byte segments: the TMA-staged z passes (wide_z = 2)
  bool tma_z16 = false;
  alignas(64) CUtensorMap tm_z16;
  // FP32 spectrum rows as [N^2][32][N/64] for the staged bin sums
  bool tma_bins = false;
  alignas(64) CUtensorMap tm_bins;
  int sm_count = 152;
  double green_coeff = 0;     // -1.5 Omega_M / (a kf^2 N^3) of the last response
  int* d_status = nullptr;
  // pinned host staging
  double* h_hist_u = nullptr;
  // history panels of the response launched ahead of the deposit (pm_nu_prepare)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool prep_pending = false;           // launched on the side stream, not yet joined
  double prep_a = 0;
  int prep_n = -1;
  const double* prep_hist = nullptr;
  std::vector<double> prep_ahist;
  double* d_hist_u2 = nullptr;         // ln a_hist of the prepared panels
  double* h_hist_u2 = nullptr;
  int* h_status = nullptr;
  // Sec. 4.4 background (PM_RELATIVISTIC): host copy uses the host R(y) table
  bool rel = false;
  RelBackground bg{};
  double* d_rtab = nullptr;
  double* d_icheb = nullptr;           // Chebyshev pieces of I(x)
  // history owned by the context (pm_history_set, pm_step): P_M^{1/2} rows and
  // their scale factors, and P_nu^{1/2} of the last step (two buffers, swapped)
  double* d_hist_own = nullptr;        // [n_hist_max][nk]
  std::vector<double> own_a;
  double* d_prev[2] = {nullptr, nullptr};
  int prev_cur = 0;
  bool have_prev = false;
  // state
  bool deposited = false, deposit_grid_valid = false, have_response = false, have_kick = false;
  bool power_set = false;         // bins replaced by pm_set_power (no spectrum behind them)
  bool counts_dirty = true;       // row counts hold a direct row sort's values (a batched kick clears them)
  int wide_y = -1, wide_z = -1, part_cps = 16;   // tuning (pm_autotune)
  int gather_rows = 0;                            // tuning: gather in the sort's row order
  bool perm_valid = false;                        // the last deposit's sort wrote perm
  bool inv_valid = false;                         // the last deposit's sort wrote inv
  int* d_inv = nullptr;                           // gather_rows 2: sorted slot of each particle
  void* d_accs = nullptr;                         // gather_rows 2: [npart][4] forces by sorted slot
  const void* dep_pos = nullptr;                  // positions of the last deposit
  double* d_bins_lattice = nullptr;   // [2][nk] lattice count / ksum, restored after pm_set_power
  float* d_X = nullptr;           // [nk][12] surrogate features
  float* d_lnR = nullptr;         // [nk] surrogate output
  double a_response = 0;
  int64_t bytes = 0;
  std::vector<long long> thr;
  std::string err;
  // per-stage timing: pending (stage, start, stop) event triples
  bool timing = false;
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> spare;
  double st_ms[PM_NSTAGES] = {};
  int64_t st_launch[PM_NSTAGES] = {}, st_calls[PM_NSTAGES] = {};
};

namespace {

int fail(pm_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(pm_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_check(pm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PM_OK;
  return fail(c, PM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Host-side fault injection for tests: NUPM_FAIL_ALLOC_AT=k makes the k-th
// device allocation of pm_init report failure.
int g_alloc_counter = 0;

int dalloc(pm_ctx* c, void** p, size_t bytes, const char* what) {
  ++g_alloc_counter;
  const char* inj = getenv("NUPM_FAIL_ALLOC_AT");
  if (inj && atoi(inj) == g_alloc_counter)
    return fail(c, PM_ERR_ALLOC, "allocation of %s (%zu bytes) failed (injected)", what, bytes);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, PM_ERR_ALLOC, "cudaMalloc of %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
  }
  c->bytes += (int64_t)bytes;
  return PM_OK;
}

double hubble(const pm_ctx* c, double a) {
  if (c->rel) return sqrt(rel_e2(a, c->bg));
  return sqrt(c->omega_m / (a * a * a) + c->omega_l);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_q (long double).
void gauss_legendre(int q, double* x, double* w) {
  const long double pi = acosl(-1.0L);
  for (int i = 0; i < q; ++i) {
    long double z = cosl(pi * (i + 0.75L) / (q + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1; }
      dp = q * (z * p1 - p0) / (z * z - 1);
      const long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    x[i] = (double)(-z);
    w[i] = (double)(2 / ((1 - z * z) * dp * dp));
  }
}

// int_{u0}^{u1} f(u) du by 16-point Gauss-Legendre on panels of width <= 1/8.
template <class F>
double integrate_u(double u0, double u1, F f) {
  static double gx[16], gw[16];
  static bool init = false;
  if (!init) {
    gauss_legendre(16, gx, gw);
    init = true;
  }
  if (u1 == u0) return 0.0;
  const int np = (int)ceil(fabs(u1 - u0) * 8.0) + 1;
  const double h = (u1 - u0) / np;
  double s = 0;
  for (int p = 0; p < np; ++p) {
    const double lo = u0 + p * h;
    double ps = 0;
    for (int i = 0; i < 16; ++i) ps += gw[i] * f(lo + 0.5 * h * (gx[i] + 1));
    s += 0.5 * h * ps;
  }
  return s;
}

// Adaptive Gauss-Legendre bisection: a panel's 16-point value is replaced by
// the sum over its halves until the two agree to tol (absolute).
template <class F>
double gl16_panel(F f, double a, double b, const double* gx, const double* gw) {
  const double h = 0.5 * (b - a), m = 0.5 * (a + b);
  double s = 0.0;
  for (int i = 0; i < 16; ++i) s += gw[i] * f(m + h * gx[i]);
  return s * h;
}
template <class F>
double gl16_adapt(F f, double a, double b, double whole, double tol, int depth, const double* gx, const double* gw) {
  const double m = 0.5 * (a + b);
  const double l = gl16_panel(f, a, m, gx, gw), r = gl16_panel(f, m, b, gx, gw);
  if (depth >= 48 || fabs(l + r - whole) <= tol) return l + r;
  return gl16_adapt(f, a, m, l, tol, depth + 1, gx, gw) + gl16_adapt(f, m, b, r, tol, depth + 1, gx, gw);
}

// The R(y) table of the Sec. 4.4 background (Eq. relativistic): at t = ln y on
// the kRel grid, ln R and d ln R / d ln y with
//   N(y)     = int_0^64 sqrt(1 + x^2/y^2) x^2 / (e^x + 1) dx,   R = N / ((3/2) zeta(3)),
//   y N'(y)  = -int_0^64 (x/y)^2 / sqrt(1 + x^2/y^2) x^2 / (e^x + 1) dx
// (x = q / T_nu0; the tail beyond x = 64 is below 1e-24 of N), each on
// [0, y] and [y, 64] by adaptive bisection to 1e-15.  Built once per process.
const double* rel_table() {
  static std::vector<double> tab;
  static std::once_flag once;
  std::call_once(once, [] {
    double gx[16], gw[16];
    gauss_legendre(16, gx, gw);
    tab.resize(2 * (size_t)kRelN);
    for (int i = 0; i < kRelN; ++i) {
      const double y = exp(kRelT0 + i * kRelH);
      auto fn = [y](double x) {
        const double r = x / y;
        return sqrt(1.0 + r * r) * x * x / (exp(x) + 1.0);
      };
      auto fd = [y](double x) {
        const double r = x / y;
        return -r * r / sqrt(1.0 + r * r) * x * x / (exp(x) + 1.0);
      };
      const double cut = y < 64.0 ? y : 64.0;
      double N = 0.0, D = 0.0;
      const double e0[2] = {0.0, cut}, e1[2] = {cut, 64.0};
      for (int k = 0; k < 2; ++k) {
        if (!(e1[k] > e0[k])) continue;
        N += gl16_adapt(fn, e0[k], e1[k], gl16_panel(fn, e0[k], e1[k], gx, gw), 1e-15, 0, gx, gw);
        D += gl16_adapt(fd, e0[k], e1[k], gl16_panel(fd, e0[k], e1[k], gx, gw), 1e-15, 0, gx, gw);
      }
      tab[2 * (size_t)i] = log(N / (1.5 * kRelZeta3));
      tab[2 * (size_t)i + 1] = D / N;
    }
  });
  return tab.data();
}

// s(u) table on u in [ln a_i, u_max], spacing 1/512: values and ds/du = 1/(a^2 H).
int build_s_table(pm_ctx* c, double u_max) {
  const double u0 = log(c->a_init);
  const double h = 1.0 / 512.0;
  int n = (int)ceil((u_max - u0) / h) + 2;
  if (n < 4) n = 4;
  std::vector<double> t(2 * (size_t)n);
  double gx[8], gw[8];
  gauss_legendre(8, gx, gw);
  double s = 0, comp = 0;   // Kahan-compensated running sum
  for (int i = 0; i < n; ++i) {
    const double u = u0 + i * h;
    const double a = exp(u);
    if (i > 0) {
      const double lo = u - h;
      double cell = 0;
      for (int k = 0; k < 8; ++k) {
        const double uu = lo + 0.5 * h * (gx[k] + 1);
        const double aa = exp(uu);
        cell += gw[k] / (aa * aa * hubble(c, aa));
      }
      cell *= 0.5 * h;
      const double y = cell - comp;
      const double tt = s + y;
      comp = (tt - s) - y;
      s = tt;
    }
    t[2 * i] = s;
    t[2 * i + 1] = 1.0 / (a * a * hubble(c, a));
  }
  if (c->d_stab) cudaFree(c->d_stab);
  c->d_stab = nullptr;
  if (cudaMalloc((void**)&c->d_stab, t.size() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PM_ERR_ALLOC, "s-table allocation failed");
  }
  if (cudaMemcpy(c->d_stab, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, PM_ERR_CUDA, "s-table upload failed");
  c->n_stab = n;
  c->stab_u0 = u0;
  c->stab_h = h;
  c->stab_umax = u0 + (n - 2) * h;
  return PM_OK;
}

template <typename T>
int upload_tables(pm_ctx* c) {
  const int n = c->n, m = c->m;
  const long double pi = acosl(-1.0L);
  // twiddles W_N^k (k < N) and W_M^k (k < M), forward sign
  std::vector<T> twn(2 * (size_t)n), twm(2 * (size_t)m);
  for (int k = 0; k < n; ++k) {
    const long double t = -2.0L * pi * k / n;
    twn[2 * k] = (T)cosl(t);
    twn[2 * k + 1] = (T)sinl(t);
  }
  for (int k = 0; k < m; ++k) {
    const long double t = -2.0L * pi * k / m;
    twm[2 * k] = (T)cosl(t);
    twm[2 * k + 1] = (T)sinl(t);
  }
  // 4-point gradient multiplier per index (signed frequency), 0 at Nyquist
  std::vector<T> dt(n), wt(n);
  for (int i = 0; i < n; ++i) {
    const int f = i < n / 2 ? i : i - n;
    const long double th = 2.0L * pi * f / n;
    long double d = (8.0L * sinl(th) - sinl(2.0L * th)) / (6.0L * (long double)c->delta);
    if (i == n / 2 || i == 0) d = 0;
    dt[i] = (T)d;
    const long double x = pi * f / n;
    const long double sc = f == 0 ? 1.0L : sinl(x) / x;
    wt[i] = (T)(1.0L / (sc * sc * sc * sc));
  }
  cudaError_t e = cudaSuccess;
  e = cudaMemcpy(c->tw_n, twn.data(), twn.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->tw_m, twm.data(), twm.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_dtab, dt.data(), dt.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_wtab, wt.data(), wt.size() * sizeof(T), cudaMemcpyHostToDevice);
  return cuda_check(c, e, "table upload");
}

cudaEvent_t take_event(pm_ctx* c) {
  if (!c->spare.empty()) {
    cudaEvent_t e = c->spare.back();
    c->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Stage scope: records an event pair around the launches of one stage when
// timing is on, and counts the stage's kernel launches.
struct Stage {
  pm_ctx* c;
  int stage;
  cudaEvent_t a = nullptr;
  Stage(pm_ctx* ctx, int st, int launches) : c(ctx), stage(st) {
    c->st_launch[st] += launches;
    c->st_calls[st] += 1;
    if (c->timing) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Stage() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->pending.push_back({stage, a, b});
    }
  }
};

void drain_timing(pm_ctx* c) {
  for (auto& r : c->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->st_ms[r.stage] += ms;
    c->spare.push_back(r.a);
    c->spare.push_back(r.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

// Encode a 4-D tensor map over a packed complex field array [F][N][N][M]
// (x2 fastest) with a box of w x2-columns by `box` elements along y or z.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

// The FP32 packed spectrum [N^2 rows][M] viewed as [rows][32 lanes][E = M / 32]
// 8-byte elements; box = one whole row, swizzle span = E * 8 bytes.
int encode_bins_map(pm_ctx* c) {
  const auto encode = tensor_map_encoder();
  if (!encode) return fail(c, PM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t E = (cuuint64_t)c->m / 32;
  cuuint64_t dims[3] = {E, 32, (cuuint64_t)c->n * c->n};
  cuuint64_t strides[2] = {E * 8, (cuuint64_t)c->m * 8};
  cuuint32_t boxd[3] = {(cuuint32_t)E, 32u, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  // the swizzle span equals a lane's segment (E * 8 bytes), so the box lands densely
  const CUtensorMapSwizzle sw = E == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : E == 8 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : E == 4 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUresult r = encode(&c->tm_bins, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, c->spec, dims, strides, boxd, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PM_OK;
}

int encode_col_map(pm_ctx* c, CUtensorMap* map, void* base, int fields, bool along_z, int w) {
  const auto encode = tensor_map_encoder();
  if (!encode) return fail(c, PM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int n = c->n, m = c->m;
  const bool f64 = c->fp64;
  const int box = n < 256 ? n : 256;
  const cuuint64_t e0 = f64 ? 2 * (cuuint64_t)m : (cuuint64_t)m;   // elements of 8 bytes
  cuuint64_t dims[4] = {e0, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)fields};
  cuuint64_t strides[3] = {e0 * 8, e0 * 8 * n, e0 * 8 * n * n};
  cuuint32_t boxd[4] = {(cuuint32_t)(f64 ? 2 * w : w), along_z ? 1u : (cuuint32_t)box,
                        along_z ? (cuuint32_t)box : 1u, 1u};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, base,
                            dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PM_OK;
}

GridArgs grid_args(const pm_ctx* c) {
  GridArgs g;
  g.wide_y = c->wide_y;
  g.wide_z = c->wide_z;
  g.part_ctas_per_sm = c->part_cps;
  g.fd_grad = !(c->p.flags & (PM_SPECTRAL_GRADIENT | PM_FUSED_GATHER | PM_TMA_COLUMNS));
  g.n = c->n;
  g.np = c->np;
  g.box = c->box;
  g.delta = c->delta;
  g.scale = (double)c->n * c->n * c->n / ((double)c->np * 281474976710656.0);   // N^3 / (Np 2^48)
  g.spec = c->spec;
  g.g = c->g;
  g.field_elems = c->field_elems;
  g.tw_n = c->tw_n;
  g.tw_m = c->tw_m;
  g.status = c->d_status;
  g.gtab = c->d_gtab;
  g.dtab = c->d_dtab;
  g.wtab = (c->p.flags & PM_DECONV_CIC) ? c->d_wtab : nullptr;
  g.plane0 = c->d_plane0;
  g.row_count = c->d_rowc;
  g.row_start = c->d_rows;
  g.row_cursor = c->d_rowcur;
  g.scan_tot = c->d_scantot;
  g.perm = ((c->p.flags & PM_FUSED_GATHER) || c->gather_rows == 1) ? c->d_perm : nullptr;
  g.inv = c->gather_rows == 2 ? c->d_inv : nullptr;
  g.bins_in_z = !c->fp64 && c->tma_z16 && c->wide_z == 2 && c->nk <= 256;
  g.bin_thr = c->d_thr;
  g.bin_inv_lr = c->bin_inv_lr;
  g.bin_nk = c->nk;
  g.bin_partials = c->d_partials;
  g.accs = c->d_accs;
  g.gather_rows = c->gather_rows;
  g.rec = c->d_rec;
  g.tmap_spec_y = c->tma ? &c->tm_spec_y : nullptr;
  g.tmap_spec_z = c->tma ? &c->tm_spec_z : nullptr;
  g.tmap_g_y = c->tma ? &c->tm_g_y : nullptr;
  g.tmap_z16 = c->tma_z16 ? &c->tm_z16 : nullptr;
  g.tmap_bins = c->tma_bins ? &c->tm_bins : nullptr;
  g.sm_count = c->sm_count;
  g.fac = c->d_fac;
  g.fac_inv_du = (float)((kFacTable - 1) / (0.5 * log((double)c->n2max)));
  g.green_coeff = (float)c->green_coeff;
  return g;
}

void release(pm_ctx* c) {
  void* ptrs[] = {c->d_bins_lattice, c->d_X, c->d_lnR,
                  c->spec, c->g, c->tw_n, c->tw_m, c->d_thr, c->d_partials, c->d_bins, c->d_pi, c->d_ti,
                  c->d_stab, c->d_hist_u, c->d_gl, c->d_parts, c->d_R, c->d_pnu, c->d_pm, c->d_rlist, c->d_gtab,
                  c->d_dtab, c->d_wtab, c->d_plane0, c->d_fac, c->d_rowc, c->d_rows, c->d_rowcur,
                  c->d_scantot, c->d_perm, c->d_rec, c->d_status, c->d_hist_u2, c->d_rtab, c->d_icheb, c->d_hist_own,
                  c->d_prev[0], c->d_prev[1], c->d_inv, c->d_accs};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_hist_u) cudaFreeHost(c->h_hist_u);
  if (c->h_hist_u2) cudaFreeHost(c->h_hist_u2);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->h_status) cudaFreeHost(c->h_status);
  for (auto& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->spare) cudaEventDestroy(e);
}

bool finite_pos(double x) { return isfinite(x) && x > 0; }

// Species masses of a problem statement (Sec. 2.1): the listed masses, or
// m_nu_total shared equally; Omega_nu from the total mass when not given.
void species_setup(const pm_params& p, double (&ms)[3], int& ns, double& mtot, double& onu) {
  mtot = p.m_nu_total_eV;
  ns = (mtot > 0) ? p.n_species : 0;
  ms[0] = ms[1] = ms[2] = 0.0;
  if (ns > 0) {
    double sum = 0;
    for (int i = 0; i < ns; ++i) sum += p.m_nu_eV[i] > 0 ? p.m_nu_eV[i] : 0;
    if (sum > 0) {
      for (int i = 0; i < ns; ++i) ms[i] = p.m_nu_eV[i] > 0 ? p.m_nu_eV[i] : 0;
      mtot = sum;
    } else {
      for (int i = 0; i < ns; ++i) ms[i] = mtot / ns;
    }
  }
  onu = p.omega_nu < 0 ? mtot / (kOmegaNuEv * p.h * p.h) : p.omega_nu;
  if (ns == 0) onu = p.omega_nu > 0 ? p.omega_nu : 0.0;
}

int n_massive_of(const double* ms, int ns, double onu) {
  int k = 0;
  for (int i = 0; i < ns && onu > 0; ++i) k += ms[i] > 0 ? 1 : 0;
  return k;
}

// The Sec. 4.4 background of species with masses m[s] and weights w[s]
// (Omega_nu,s = Omega_nu w[s]): massive species with the energy density of
// Eq. relativistic, radiation (photons and the massless of three species),
// Lambda closing the universe at a = 1.
void fill_background(const pm_params& p, const double* m, const double* w, int ns, double onu, int n_massive,
                     RelBackground& B) {
  B.tab = rel_table();
  B.om_r = kOmegaGammaH2 / (p.h * p.h) * (1.0 + (kNuSpeciesTotal - n_massive) * nu_to_gamma());
  B.om_cdm = p.omega_cdm;
  double nu_today = 0.0;
  B.ns = 0;
  if (ns > 0 && onu > 0) {
    B.ns = ns;
    for (int s = 0; s < ns; ++s) {
      B.om_nu[s] = onu * w[s];
      B.y1[s] = m[s] / kTnu0eV;
      nu_today += B.om_nu[s] * nu_rho_ratio(B.y1[s], B.tab);
    }
  } else {
    B.om_cdm += onu;   // Omega_nu without a massive species: clustering matter
    nu_today = onu;
  }
  B.om_lam = 1.0 - p.omega_cdm - nu_today - B.om_r;
}

}  // namespace

extern "C" {

void pm_default_params(pm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->ngrid = 32;
  p->npart = 32 * 32 * 32;
  p->box = 256.0;
  p->particle_mass = 1.0;
  p->omega_cdm = 0.3;
  p->omega_nu = 0.0;
  p->h = 0.7;
  p->a_init = 0.02;
  p->n_kbins = 32;
  p->n_hist_max = 128;
  p->precision = PM_FP64;
  p->iters = 1;
  p->quad_nodes = 8;
}

int pm_init(const pm_params* params, const double* sqrtPnu_init, const double* theta_over_delta_init,
            void* cuda_stream, pm_ctx** out) {
  if (!out) return PM_ERR_INVALID;
  *out = nullptr;
  if (!params) return PM_ERR_INVALID;
  pm_ctx* c = new pm_ctx();
  c->p = *params;
  const pm_params& p = *params;
  int rc = PM_OK;
  auto bad = [&](int code, const char* msg) {
    c->err = msg;
    rc = code;
  };
  const int n = p.ngrid;
  const bool pow2 = n >= 16 && n <= 1024 && (n & (n - 1)) == 0;
  if (!pow2 && n != 192) bad(PM_ERR_UNSUPPORTED, "ngrid must be a power of two in [16, 1024] or 192");
  else if (!pow2 && (p.flags & (PM_TMA_COLUMNS | PM_FUSED_GATHER)))
    bad(PM_ERR_UNSUPPORTED, "PM_TMA_COLUMNS / PM_FUSED_GATHER need a power-of-two grid");
  else if (p.npart < 1) bad(PM_ERR_INVALID, "npart must be >= 1");
  else if (p.npart > 0x7fffffffLL) bad(PM_ERR_INVALID, "npart must be < 2^31");
  else if (!finite_pos(p.box)) bad(PM_ERR_INVALID, "box must be finite and > 0");
  else if (!finite_pos(p.particle_mass)) bad(PM_ERR_INVALID, "particle_mass must be finite and > 0");
  else if (!(isfinite(p.omega_cdm) && p.omega_cdm > 0)) bad(PM_ERR_INVALID, "omega_cdm must be > 0");
  else if (!finite_pos(p.h)) bad(PM_ERR_INVALID, "h must be > 0");
  else if (!(isfinite(p.m_nu_total_eV) && p.m_nu_total_eV >= 0)) bad(PM_ERR_RANGE, "m_nu_total_eV must be >= 0");
  else if (p.n_species < 0 || p.n_species > 3) bad(PM_ERR_INVALID, "n_species must be 0..3");
  else if (!(isfinite(p.a_init) && p.a_init > 0 && p.a_init <= 1)) bad(PM_ERR_RANGE, "a_init must be in (0, 1]");
  else if (p.n_kbins < 1 || p.n_kbins > 1024) bad(PM_ERR_INVALID, "n_kbins must be 1..1024");
  else if (p.n_hist_max < 0 || p.n_hist_max > kMaxPanels - 64) bad(PM_ERR_INVALID, "n_hist_max must be 0..256");
  else if (p.precision != PM_FP64 && p.precision != PM_FP32) bad(PM_ERR_INVALID, "precision must be PM_FP64 or PM_FP32");
  else if (p.iters < 1 || p.iters > 16) bad(PM_ERR_INVALID, "iters must be 1..16");
  else if (p.quad_nodes < 2 || p.quad_nodes > kMaxQuad) bad(PM_ERR_INVALID, "quad_nodes must be 2..16");
  else if (p.flags & ~(PM_I_FIT | PM_DECONV_CIC | PM_KEEP_DEPOSIT | PM_UNFUSED_DEPOSIT | PM_TMA_COLUMNS | PM_FUSED_GATHER |
                       PM_SPECTRAL_GRADIENT | PM_RELATIVISTIC | PM_IC_MULTIPOLE))
    bad(PM_ERR_INVALID, "unknown flag bits");
  if (rc != PM_OK) {
    // report through a context so pm_last_error works; caller still gets NULL
    fprintf(stderr, "pm_init: %s\n", c->err.c_str());
    delete c;
    return rc;
  }
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->fp64 = p.precision == PM_FP64;
  c->n = n;
  c->m = n / 2;
  c->nk = p.n_kbins;
  c->np = p.npart;
  c->box = p.box;
  c->delta = p.box / n;
  c->kf = 2.0 * M_PI / p.box;
  c->quad = p.quad_nodes;
  c->iters = p.iters;
  c->a_init = p.a_init;
  // neutrinos (Sec. 2.1): Omega_nu from the total mass when not given
  double mtot = 0.0, onu = 0.0;
  int ns = 0;
  double ms[3] = {0, 0, 0};
  species_setup(p, ms, ns, mtot, onu);
  if (!(isfinite(onu) && onu >= 0)) {
    fprintf(stderr, "pm_init: bad omega_nu\n");
    delete c;
    return PM_ERR_RANGE;
  }
  c->omega_nu = onu;
  c->omega_m = p.omega_cdm + onu;
  c->omega_l = 1.0 - c->omega_m;
  c->f_nu = onu / c->omega_m;
  // massless species carry no weight; a species of mass 0 is skipped
  // Species of equal mass and identical initial conditions give identical
  // responses: merge them into one species carrying their summed weight.
  const int nkb = p.n_kbins;
  std::vector<std::vector<double>> sp_pi, sp_ti;
  double wsum = 0;
  for (int i = 0; i < ns; ++i) wsum += ms[i];
  int used = 0;
  for (int i = 0; i < ns; ++i) {
    if (ms[i] <= 0) continue;
    std::vector<double> pi(nkb, 0.0), ti(nkb, 0.0);
    for (int b = 0; b < nkb; ++b) {
      if (sqrtPnu_init) pi[b] = sqrtPnu_init[(size_t)i * nkb + b];
      if (theta_over_delta_init) ti[b] = theta_over_delta_init[(size_t)i * nkb + b];
      if (!isfinite(pi[b]) || !isfinite(ti[b])) {
        fprintf(stderr, "pm_init: non-finite neutrino initial condition\n");
        delete c;
        return PM_ERR_INVALID;
      }
    }
    int match = -1;
    for (int j = 0; j < used; ++j)
      if (c->mass[j] == ms[i] && sp_pi[j] == pi && sp_ti[j] == ti) match = j;
    if (match >= 0) {
      c->wsp[match] += ms[i] / wsum;
    } else {
      c->mass[used] = ms[i];
      c->wsp[used] = ms[i] / wsum;
      sp_pi.push_back(pi);
      sp_ti.push_back(ti);
      ++used;
    }
  }
  c->ns = used;
  if (p.flags & PM_RELATIVISTIC) {
    c->rel = true;
    fill_background(p, c->mass, c->wsp, c->ns, onu, n_massive_of(ms, ns, onu), c->bg);
  }
  c->n2max = 3LL * (n / 2) * (n / 2);
  c->field_elems = (int64_t)n * n * (n / 2);
  c->cplx = c->fp64 ? 16 : 8;
  const size_t real = c->fp64 ? 8 : 4;
  c->nblk_bins = 152 * 8;

  int nspec = c->ns > 0 ? c->ns : 1;
  g_alloc_counter = 0;
  const size_t fbytes = (size_t)c->field_elems * c->cplx;
  if (rc == PM_OK) rc = dalloc(c, &c->spec, fbytes, "spectrum");
  if (rc == PM_OK) rc = dalloc(c, &c->g, 3 * fbytes, "force fields");
  if (rc == PM_OK) rc = dalloc(c, &c->tw_n, (size_t)n * c->cplx, "twiddles N");
  if (rc == PM_OK) rc = dalloc(c, &c->tw_m, (size_t)(n / 2) * c->cplx, "twiddles M");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_thr, (size_t)(c->nk + 1) * sizeof(int), "bin thresholds");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_partials, (size_t)c->nblk_bins * 2 * c->nk * sizeof(double), "bin partials");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_bins, 3 * (size_t)c->nk * sizeof(double), "bins");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_bins_lattice, 2 * (size_t)c->nk * sizeof(double), "lattice bins");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_X, 12 * (size_t)c->nk * sizeof(float), "surrogate features");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_lnR, (size_t)c->nk * sizeof(float), "surrogate output");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_pi, (size_t)nspec * c->nk * sizeof(double), "nu ICs");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_ti, (size_t)nspec * c->nk * sizeof(double), "nu theta ICs");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_hist_u, (size_t)(p.n_hist_max + 1) * sizeof(double), "history ln a");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_hist_u2, (size_t)(p.n_hist_max + 1) * sizeof(double), "history ln a");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_gl, 2 * kMaxQuad * sizeof(double), "quadrature");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_parts, (size_t)nspec * c->nk * kNuChunks * 3 * sizeof(double), "response parts");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_rlist, (2 * (size_t)c->nk + 1) * sizeof(double), "ratio list");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_R, (size_t)c->nk * sizeof(double), "ratio");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_pnu, (size_t)c->nk * sizeof(double), "P_nu");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_pm, (size_t)c->nk * sizeof(double), "P_M");
  if (rc == PM_OK) rc = dalloc(c, &c->d_gtab, (size_t)(c->n2max + 1) * real, "Green table");
  if (rc == PM_OK) rc = dalloc(c, &c->d_dtab, (size_t)n * real, "gradient table");
  if (rc == PM_OK) rc = dalloc(c, &c->d_wtab, (size_t)n * real, "deconvolution table");
  if (rc == PM_OK) rc = dalloc(c, &c->d_plane0, (size_t)n * n * c->cplx, "Green plane x2=0");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_fac, kFacTable * sizeof(float), "fac table");
  const size_t nrow1 = (size_t)n * n + 1;
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_rowc, nrow1 * sizeof(int), "row counts");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_rows, nrow1 * sizeof(int), "row starts");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_rowcur, nrow1 * sizeof(int), "row cursors");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_scantot, 2048 * sizeof(int), "scan totals");
  if (rc == PM_OK && !(p.flags & PM_UNFUSED_DEPOSIT))
    rc = dalloc(c, (void**)&c->d_perm, (size_t)c->np * sizeof(int), "row permutation");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_rec, (size_t)c->np * sizeof(unsigned long long), "sorted records");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_status, sizeof(int), "status");
  if (rc == PM_OK)
    rc = dalloc(c, (void**)&c->d_hist_own, (size_t)(p.n_hist_max > 0 ? p.n_hist_max : 1) * c->nk * sizeof(double),
                "stored history");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_prev[0], (size_t)c->nk * sizeof(double), "previous P_nu");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_prev[1], (size_t)c->nk * sizeof(double), "previous P_nu");
  if (rc == PM_OK) rc = dalloc(c, (void**)&c->d_icheb, (size_t)kISeg * kICoef * sizeof(double), "I(x) table");
  if (rc == PM_OK) {
    launch_I_table(c->d_icheb, c->stream);
    rc = cuda_check(c, cudaGetLastError(), "I(x) table");
    // other streams (the side stream, batched kicks) read it without an event
    if (rc == PM_OK) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "I(x) table");
  }
  if (rc == PM_OK && c->rel) {
    rc = dalloc(c, (void**)&c->d_rtab, 2 * (size_t)kRelN * sizeof(double), "relativistic background table");
    if (rc == PM_OK)
      rc = cuda_check(c, cudaMemcpy(c->d_rtab, c->bg.tab, 2 * (size_t)kRelN * sizeof(double), cudaMemcpyHostToDevice),
                      "background table upload");
  }
  if (rc == PM_OK && (cudaMallocHost((void**)&c->h_hist_u2, (size_t)(p.n_hist_max + 1) * sizeof(double)) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = fail(c, PM_ERR_ALLOC, "side stream or pinned history allocation failed");
  if (rc == PM_OK && cudaMallocHost((void**)&c->h_hist_u, (size_t)(p.n_hist_max + 1) * sizeof(double)) != cudaSuccess)
    rc = fail(c, PM_ERR_ALLOC, "pinned host allocation failed");
  if (rc == PM_OK && cudaMallocHost((void**)&c->h_status, sizeof(int)) != cudaSuccess)
    rc = fail(c, PM_ERR_ALLOC, "pinned host allocation failed");
  if (rc == PM_OK) rc = c->fp64 ? upload_tables<double>(c) : upload_tables<float>(c);
  if (rc == PM_OK) {
    // bin thresholds T_b = ceil((e_b L / 2 pi)^2), e_b log-spaced on [kmin, kmax];
    // mode n^2 is in bin b iff T_b <= n^2 < T_{b+1}
    c->thr.resize(c->nk + 1);
    bin_thresholds(n, c->nk, c->thr.data());
    std::vector<int> t32(c->thr.begin(), c->thr.end());   // T_nk <= 3 N^2 / 4 + 1 fits int32
    c->bin_inv_lr = (float)(c->nk / (2.0 * bin_log_ratio(n)));
    rc = cuda_check(c, cudaMemcpy(c->d_thr, t32.data(), t32.size() * sizeof(int), cudaMemcpyHostToDevice),
                    "bin threshold upload");
  }
  if (rc == PM_OK) {
    std::vector<double> gl(2 * kMaxQuad, 0.0);
    gauss_legendre(c->quad, gl.data(), gl.data() + kMaxQuad);
    rc = cuda_check(c, cudaMemcpy(c->d_gl, gl.data(), gl.size() * sizeof(double), cudaMemcpyHostToDevice),
                    "quadrature upload");
  }
  if (rc == PM_OK) {
    // neutrino ICs per (merged) species
    std::vector<double> pi((size_t)nspec * c->nk, 0.0), ti((size_t)nspec * c->nk, 0.0);
    for (int j = 0; j < c->ns; ++j)
      for (int b = 0; b < c->nk; ++b) {
        pi[(size_t)j * c->nk + b] = sp_pi[j][b];
        ti[(size_t)j * c->nk + b] = sp_ti[j][b];
      }
    rc = cuda_check(c, cudaMemcpy(c->d_pi, pi.data(), pi.size() * sizeof(double), cudaMemcpyHostToDevice), "IC upload");
    if (rc == PM_OK)
      rc = cuda_check(c, cudaMemcpy(c->d_ti, ti.data(), ti.size() * sizeof(double), cudaMemcpyHostToDevice), "IC upload");
  }
  if (rc == PM_OK) rc = build_s_table(c, 0.0 > log(c->a_init) ? 0.0 : log(c->a_init) + 1.0);
  if (rc == PM_OK) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (p.flags & PM_TMA_COLUMNS) {
      const int w = c->fp64 ? 4 : 8;   // 64-byte row segments
      rc = encode_col_map(c, &c->tm_spec_y, c->spec, 1, false, w);
      if (rc == PM_OK) rc = encode_col_map(c, &c->tm_spec_z, c->spec, 1, true, w);
      if (rc == PM_OK) rc = encode_col_map(c, &c->tm_g_y, c->g, 3, false, w);
      c->tma = rc == PM_OK;
    }
    // TMA-staged z passes (a tuning choice, power-of-two grids from 256 on):
    // without the driver's encoder they are simply not offered
    if (rc == PM_OK && pow2 && c->n >= 256) {
      const std::string keep = c->err;
      c->tma_z16 = encode_col_map(c, &c->tm_z16, c->spec, 1, true, c->fp64 ? 8 : 16) == PM_OK;
      c->err = keep;
    }
    // TMA-staged FP32 bin sums (N / 64 modes of a row per lane: 2 .. 16)
    if (rc == PM_OK && pow2 && !c->fp64 && c->n >= 128) {
      const std::string keep = c->err;
      c->tma_bins = encode_bins_map(c) == PM_OK;
      c->err = keep;
    }
  }
  if (rc == PM_OK) {
    // mode counts and sum |k| per bin depend on the lattice only: once per context
    GridArgs g = grid_args(c);
    rc = c->fp64 ? bins_f64(g, true, c->nk, c->d_thr, c->bin_inv_lr, c->kf, c->d_partials, c->nblk_bins, c->d_bins, 0)
                 : bins_f32(g, true, c->nk, c->d_thr, c->bin_inv_lr, c->kf, c->d_partials, c->nblk_bins, c->d_bins, 0);
    if (rc == PM_OK) rc = cuda_check(c, cudaGetLastError(), "lattice bins");
    if (rc == PM_OK)
      rc = cuda_check(c, cudaMemcpy(c->d_bins_lattice, c->d_bins, 2 * (size_t)c->nk * sizeof(double),
                                    cudaMemcpyDeviceToDevice), "lattice bins copy");
  }
  if (rc == PM_OK) rc = cuda_check(c, cudaMemset(c->d_status, 0, sizeof(int)), "status init");
  if (rc == PM_OK) rc = cuda_check(c, cudaDeviceSynchronize(), "pm_init");
  if (rc != PM_OK) {
    fprintf(stderr, "pm_init: %s\n", c->err.c_str());
    release(c);
    delete c;
    return rc;
  }
  *out = c;
  return PM_OK;
}

int pm_deposit(pm_ctx* c, const void* pos) {
  if (!c) return PM_ERR_INVALID;
  if (!pos) return fail(c, PM_ERR_INVALID, "pm_deposit: pos is NULL");
  GridArgs g = grid_args(c);
  int rc = PM_OK;
  if (c->power_set) {
    rc = cuda_check(c, cudaMemcpyAsync(c->d_bins, c->d_bins_lattice, 2 * (size_t)c->nk * sizeof(double),
                                       cudaMemcpyDeviceToDevice, c->stream), "lattice bins restore");
    if (rc != PM_OK) return rc;
    c->power_set = false;
  }
  const bool unfused = (c->p.flags & PM_UNFUSED_DEPOSIT) != 0;
  const bool keep = (c->p.flags & PM_KEEP_DEPOSIT) != 0;
  if (unfused) {
    {
      Stage st(c, PM_ST_DEPOSIT, 1);
      rc = c->fp64 ? deposit_f64(g, pos, c->stream) : deposit_f32(g, pos, c->stream);
    }
    if (rc == PM_OK) {
      Stage st(c, PM_ST_FFT_X_FWD, 1);
      rc = c->fp64 ? fft_pass_f64(g, kPassXFwd, c->stream) : fft_pass_f32(g, kPassXFwd, c->stream);
    }
  } else {
    {
      Stage st(c, PM_ST_DEPOSIT, 5);
      rc = c->fp64 ? row_sort_f64(g, pos, c->stream) : row_sort_f32(g, pos, c->stream);
      c->counts_dirty = true;
    }
    if (rc == PM_OK) {
      Stage st(c, PM_ST_FFT_X_FWD, 1);
      rc = c->fp64 ? deposit_fft_x_f64(g, pos, keep, c->stream) : deposit_fft_x_f32(g, pos, keep, c->stream);
    }
  }
  const int fwd[2] = {kPassYFwd, kPassZFwd};
  const int fst[2] = {PM_ST_FFT_Y_FWD, PM_ST_FFT_Z_FWD};
  for (int i = 0; i < 2 && rc == PM_OK; ++i) {
    Stage st(c, fst[i], 1);
    rc = c->fp64 ? fft_pass_f64(g, fwd[i], c->stream) : fft_pass_f32(g, fwd[i], c->stream);
  }
  if (rc == PM_OK) {
    Stage st(c, PM_ST_BINS, 2);
    rc = c->fp64 ? bins_f64(g, false, c->nk, c->d_thr, c->bin_inv_lr, c->kf, c->d_partials, c->nblk_bins, c->d_bins + 2 * c->nk,
                            c->stream)
                 : bins_f32(g, false, c->nk, c->d_thr, c->bin_inv_lr, c->kf, c->d_partials, c->nblk_bins, c->d_bins + 2 * c->nk,
                            c->stream);
  }
  if (rc != PM_OK) return fail(c, rc, "pm_deposit: unsupported grid");
  rc = cuda_check(c, cudaGetLastError(), "pm_deposit launch");
  if (rc != PM_OK) return rc;
  c->deposited = true;
  c->deposit_grid_valid = unfused || keep;   // the fixed-point grid stays intact until pm_kick
  c->perm_valid = !unfused && g.perm != nullptr;
  c->inv_valid = !unfused && g.inv != nullptr;
  c->dep_pos = pos;
  c->have_response = false;
  c->have_kick = false;
  return PM_OK;
}

}  // extern "C"

namespace {

// Checks of a response call's arguments, history upload (ln a_j) and the s(a)
// table extension, shared by the exact and the surrogate response.
int response_prepare(pm_ctx* c, double a, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist) {
  if (!c->deposited) return fail(c, PM_ERR_ORDER, "pm_nu_response before pm_deposit");
  if (!(isfinite(a) && a >= c->a_init)) return fail(c, PM_ERR_RANGE, "a must be finite and >= a_init");
  if (n_hist < 0 || n_hist > c->p.n_hist_max) return fail(c, PM_ERR_INVALID, "n_hist outside 0..n_hist_max");
  if (n_hist > 0 && (!a_hist || !sqrtPM_hist)) return fail(c, PM_ERR_INVALID, "history pointers are NULL");
  for (int j = 0; j < n_hist; ++j) {
    if (!isfinite(a_hist[j])) return fail(c, PM_ERR_RANGE, "non-finite a_hist");
    if (j == 0 && a_hist[0] < c->a_init) return fail(c, PM_ERR_RANGE, "a_hist[0] < a_init");
    if (j > 0 && !(a_hist[j] > a_hist[j - 1])) return fail(c, PM_ERR_RANGE, "a_hist not strictly increasing");
  }
  if (n_hist > 0 && !(a_hist[n_hist - 1] < a)) return fail(c, PM_ERR_RANGE, "a_hist[n-1] must be < a");
  const double ue = log(a);
  if (ue > c->stab_umax) {
    const int rc = build_s_table(c, ue + 1.0);
    if (rc != PM_OK) return rc;
  }
  for (int j = 0; j < n_hist; ++j) c->h_hist_u[j] = log(a_hist[j]);
  if (n_hist > 0)
    return cuda_check(c, cudaMemcpyAsync(c->d_hist_u, c->h_hist_u, n_hist * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream), "history upload");
  return PM_OK;
}

// NuArgs of the surrogate kernels (bins, history, outputs).
NuArgs surrogate_args(pm_ctx* c, double a, const double* sqrtPM_hist, int32_t n_hist, double* ratio_out,
                      double* sqrtPnu_out, double* sqrtPM_out) {
  NuArgs A{};
  A.nk = c->nk;
  A.ns = c->ns;
  A.n_hist = n_hist;
  A.ngrid = c->n;
  A.a = a;
  A.ue = log(a);
  A.ui = log(c->a_init);
  A.f_nu = c->f_nu;
  A.box = c->box;
  A.bins = c->d_bins;
  A.hist_u = c->d_hist_u;
  A.hist = sqrtPM_hist;
  A.rlist = c->d_rlist;
  A.R = c->d_R;
  A.pnu = c->d_pnu;
  A.pm = c->d_pm;
  A.R_user = ratio_out;
  A.pnu_user = sqrtPnu_out;
  A.pm_user = sqrtPM_out;
  return A;
}

// Green and fac tables from the response's rlist (both response forms).
// A side-stream launch of pm_nu_prepare that no pm_nu_response consumed:
// joined into the context's stream (and dropped).
int join_prepared(pm_ctx* c) {
  if (!c->prep_pending) return PM_OK;
  c->prep_pending = false;
  return cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "side stream join");
}

// NuArgs of the exact response (bins, history, tables, outputs).
NuArgs nu_args(pm_ctx* c, double a, const double* sqrtPM_hist, int32_t n_hist, const double* sqrtPnu_prev,
               double* ratio_out, double* sqrtPnu_out, double* sqrtPM_out) {
  NuArgs A{};
  A.nk = c->nk;
  A.ns = (c->ns > 0 && c->f_nu > 0) ? c->ns : 0;
  A.n_hist = n_hist;
  A.quad = c->quad;
  A.iters = A.ns > 0 ? c->iters : 1;
  A.use_fit = (c->p.flags & PM_I_FIT) ? 1 : 0;
  A.ngrid = c->n;
  A.a = a;
  A.ue = log(a);
  A.ui = log(c->a_init);
  A.omega_m = c->omega_m;
  A.omega_l = c->omega_l;
  A.f_nu = c->f_nu;
  A.a_init = c->a_init;
  A.box = c->box;
  for (int s = 0; s < c->ns; ++s) {
    A.kappa_scale[s] = kCOverH0 * kTnu0eV / c->mass[s];
    A.w_species[s] = c->wsp[s];
  }
  A.bins = c->d_bins;
  A.hist_u = c->d_hist_u;
  A.hist = sqrtPM_hist;
  A.prev = sqrtPnu_prev;
  A.pnu_init = c->d_pi;
  A.theta_init = c->d_ti;
  A.stab = c->d_stab;
  A.n_stab = c->n_stab;
  A.stab_u0 = c->stab_u0;
  A.stab_h = c->stab_h;
  A.stab_inv_h = 1.0 / c->stab_h;
  A.gl = c->d_gl;
  A.icheb = c->d_icheb;
  // panel chunks in use: the panels are the history nodes, the graded points
  // a - ell 2^m (m >= -2) above a_i, at most log2((ln a - ln a_i) / ell) + 3 of
  // them with ell = a^2 H / kappa smallest at the largest |k| of the grid, and
  // the ends; 32 panels a chunk.  A chunk's warp strides over the panels by the
  // chunk count, so the bound sets the split of the work, not which panels count.
  {
    double kap = 0.0;
    for (int s = 0; s < c->ns; ++s) kap = A.kappa_scale[s] > kap ? A.kappa_scale[s] : kap;
    kap *= c->kf * sqrt(3.0) * 0.5 * c->n;
    int npan = (n_hist > 0 ? n_hist : 0) + 4;
    if (kap > 0.0 && A.ue > A.ui) {
      const double r = (A.ue - A.ui) * kap / (a * a * hubble(c, a));
      npan += 3 + (r > 1.0 ? (int)ceil(log2(r)) : 0);
    }
    const int ch = (npan + 31) / 32;
    A.nchunks = ch < 1 ? 1 : (ch > kNuChunks ? kNuChunks : ch);
  }
  A.parts = c->d_parts;
  A.rlist = c->d_rlist;
  A.R = c->d_R;
  A.pnu = c->d_pnu;
  A.pm = c->d_pm;
  A.R_user = ratio_out;
  A.pnu_user = sqrtPnu_out;
  A.pm_user = sqrtPM_out;
  A.rel = c->rel ? 1 : 0;
  A.ic_multipole = (c->p.flags & PM_IC_MULTIPOLE) ? 1 : 0;
  A.bg = c->bg;
  A.bg.tab = c->d_rtab;
  return A;
}

int response_tables(pm_ctx* c, double a) {
  const double coeff = -1.5 * c->omega_m / (a * c->kf * c->kf * (double)c->n * c->n * c->n);
  // FP64: the exact G(n^2) table; FP32: the fac(ln k) table (its Green values
  // are evaluated per mode by the passes that need them)
  if (c->fp64) launch_green_table(true, c->d_gtab, c->n2max, c->kf, coeff, c->f_nu, c->d_rlist, c->nk, c->stream);
  else launch_fac_table(c->d_fac, 0.5 * log((double)c->n2max), c->kf, c->f_nu, c->d_rlist, c->nk, c->stream);
  c->green_coeff = coeff;
  const int rc = cuda_check(c, cudaGetLastError(), "pm_nu_response launch");
  if (rc != PM_OK) return rc;
  c->have_response = true;
  c->a_response = a;
  return PM_OK;
}

}  // namespace

extern "C" {

int pm_nu_response(pm_ctx* c, double a, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist,
                   const double* sqrtPnu_prev, double* ratio_out, double* sqrtPnu_out, double* sqrtPM_out) {
  if (!c) return PM_ERR_INVALID;
  // panels launched by pm_nu_prepare: joined first, whatever happens next
  const bool had_prep = c->prep_pending;
  if (had_prep) {
    const int rc = cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "side stream join");
    if (rc != PM_OK) return rc;
    c->prep_pending = false;
  }
  bool use_prep = had_prep && !c->power_set && a == c->prep_a && n_hist == c->prep_n && sqrtPM_hist == c->prep_hist;
  for (int j = 0; use_prep && j < n_hist; ++j) use_prep = a_hist[j] == c->prep_ahist[j];
  if (!use_prep) {
    const int rc = response_prepare(c, a, a_hist, sqrtPM_hist, n_hist);
    if (rc != PM_OK) return rc;
  } else if (!c->deposited) {
    return fail(c, PM_ERR_ORDER, "pm_nu_response before pm_deposit");
  }
  const bool nu = c->ns > 0 && c->f_nu > 0;
  Stage stage(c, PM_ST_RESPONSE, (nu && !use_prep ? 1 : 0) + 3);   // [panels,] finish, bin list, table
  NuArgs A = nu_args(c, a, sqrtPM_hist, n_hist, sqrtPnu_prev, ratio_out, sqrtPnu_out, sqrtPM_out);
  if (use_prep) A.hist_u = c->d_hist_u2;
  if (nu && !use_prep) launch_nu_panels(A, c->stream);
  launch_nu_finish(A, c->stream);   // without neutrinos: R = 0, P_nu = 0, P_M^{1/2} = (1 - f) P_cdm^{1/2}
  return response_tables(c, a);
}

int pm_nu_prepare(pm_ctx* c, double a, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist) {
  if (!c) return PM_ERR_INVALID;
  if (c->prep_pending) return fail(c, PM_ERR_ORDER, "pm_nu_prepare twice without pm_nu_response");
  if (!(isfinite(a) && a >= c->a_init)) return fail(c, PM_ERR_RANGE, "a must be finite and >= a_init");
  if (n_hist < 0 || n_hist > c->p.n_hist_max) return fail(c, PM_ERR_INVALID, "n_hist outside 0..n_hist_max");
  if (n_hist > 0 && (!a_hist || !sqrtPM_hist)) return fail(c, PM_ERR_INVALID, "history pointers are NULL");
  for (int j = 0; j < n_hist; ++j) {
    if (!isfinite(a_hist[j])) return fail(c, PM_ERR_RANGE, "non-finite a_hist");
    if (j == 0 && a_hist[0] < c->a_init) return fail(c, PM_ERR_RANGE, "a_hist[0] < a_init");
    if (j > 0 && !(a_hist[j] > a_hist[j - 1])) return fail(c, PM_ERR_RANGE, "a_hist not strictly increasing");
  }
  if (n_hist > 0 && !(a_hist[n_hist - 1] < a)) return fail(c, PM_ERR_RANGE, "a_hist[n-1] must be < a");
  const double ue = log(a);
  if (ue > c->stab_umax) {
    const int rc = build_s_table(c, ue + 1.0);
    if (rc != PM_OK) return rc;
  }
  c->prep_a = a;
  c->prep_n = n_hist;
  c->prep_hist = sqrtPM_hist;
  c->prep_ahist.assign(a_hist ? a_hist : &a, a_hist ? a_hist + n_hist : &a);
  for (int j = 0; j < n_hist; ++j) c->h_hist_u2[j] = log(a_hist[j]);
  int rc = cuda_check(c, cudaEventRecord(c->ev_fork, c->stream), "side stream fork");
  if (rc == PM_OK) rc = cuda_check(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "side stream fork");
  if (rc != PM_OK) return rc;
  if (n_hist > 0)
    rc = cuda_check(c, cudaMemcpyAsync(c->d_hist_u2, c->h_hist_u2, n_hist * sizeof(double), cudaMemcpyHostToDevice,
                                       c->side), "history upload");
  if (rc == PM_OK && c->ns > 0 && c->f_nu > 0) {
    cudaEvent_t t0 = nullptr;
    if (c->timing) {
      t0 = take_event(c);
      cudaEventRecord(t0, c->side);
    }
    NuArgs A = nu_args(c, a, sqrtPM_hist, n_hist, nullptr, nullptr, nullptr, nullptr);
    A.hist_u = c->d_hist_u2;
    A.bins = c->d_bins_lattice;   // |k| of the bins: the lattice's (the deposit may rewrite d_bins meanwhile)
    launch_nu_panels(A, c->side);
    c->st_launch[PM_ST_RESPONSE] += 1;
    if (t0) {
      cudaEvent_t t1 = take_event(c);
      cudaEventRecord(t1, c->side);
      c->pending.push_back({PM_ST_RESPONSE, t0, t1});
    }
    rc = cuda_check(c, cudaGetLastError(), "pm_nu_prepare launch");
  }
  if (rc == PM_OK) rc = cuda_check(c, cudaEventRecord(c->ev_join, c->side), "side stream join");
  if (rc == PM_OK) c->prep_pending = true;
  return rc;
}

int pm_response_features(pm_ctx* c, double a, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist,
                         float* X) {
  if (!c) return PM_ERR_INVALID;
  if (!X) return fail(c, PM_ERR_INVALID, "pm_response_features: X is NULL");
  int rc = join_prepared(c);
  if (rc == PM_OK) rc = response_prepare(c, a, a_hist, sqrtPM_hist, n_hist);
  if (rc != PM_OK) return rc;
  NuArgs A = surrogate_args(c, a, sqrtPM_hist, n_hist, nullptr, nullptr, nullptr);
  launch_nu_features(A, c->p.m_nu_total_eV, c->omega_nu, X, c->stream);
  return cuda_check(c, cudaGetLastError(), "pm_response_features launch");
}

int pm_nu_response_mlp(pm_ctx* c, pm_mlp* mlp, double a, const double* a_hist, const double* sqrtPM_hist,
                       int32_t n_hist, double* ratio_out, double* sqrtPnu_out, double* sqrtPM_out) {
  if (!c) return PM_ERR_INVALID;
  if (join_prepared(c) != PM_OK) return PM_ERR_CUDA;
  if (!mlp) return fail(c, PM_ERR_INVALID, "pm_nu_response_mlp: mlp is NULL");
  if (mlp_inputs(mlp) != PM_MLP_FEATURES) return fail(c, PM_ERR_INVALID, "surrogate needs 12 input features");
  int rc = response_prepare(c, a, a_hist, sqrtPM_hist, n_hist);
  if (rc != PM_OK) return rc;
  NuArgs A = surrogate_args(c, a, sqrtPM_hist, n_hist, ratio_out, sqrtPnu_out, sqrtPM_out);
  Stage stage(c, PM_ST_RESPONSE, (c->ns > 0 && c->f_nu > 0) ? 4 : 2);
  if (c->ns > 0 && c->f_nu > 0) {
    launch_nu_features(A, c->p.m_nu_total_eV, c->omega_nu, c->d_X, c->stream);
    rc = mlp_forward_on(mlp, c->d_X, c->nk, c->d_lnR, c->stream);
    if (rc != PM_OK) return fail(c, rc, "surrogate forward launch failed");
    launch_nu_from_lnR(A, c->d_lnR, c->stream);
  } else {
    A.ns = 0;
    A.iters = 1;
    A.parts = c->d_parts;
    A.pnu_init = c->d_pi;
    launch_nu_response(A, c->stream);   // R = 0 as the exact path
  }
  return response_tables(c, a);
}

int pm_set_power(pm_ctx* c, const double* count, const double* ksum, const double* psum) {
  if (!c) return PM_ERR_INVALID;
  if (!count || !ksum || !psum) return fail(c, PM_ERR_INVALID, "pm_set_power: NULL array");
  const int nk = c->nk;
  std::vector<double> h(3 * (size_t)nk);
  for (int b = 0; b < nk; ++b) {
    if (!(count[b] >= 0.0 && isfinite(count[b]) && isfinite(ksum[b]) && isfinite(psum[b]) && psum[b] >= 0.0) ||
        (count[b] > 0.0 && !(ksum[b] > 0.0)))
      return fail(c, PM_ERR_RANGE, "pm_set_power: counts, ksum and psum must be finite, >= 0 (ksum > 0 if count > 0)");
    h[b] = count[b];
    h[nk + b] = ksum[b];
    h[2 * nk + b] = psum[b];
  }
  int rc = cuda_check(c, cudaMemcpyAsync(c->d_bins, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream), "pm_set_power upload");
  if (rc == PM_OK) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "pm_set_power sync");
  if (rc != PM_OK) return rc;
  c->deposited = true;
  c->power_set = true;
  c->have_response = false;
  return PM_OK;
}

int pm_kick(pm_ctx* c, const void* pos, void* vel, double a, double kick_factor, void* acc_out) {
  if (!c) return PM_ERR_INVALID;
  if (!pos || !vel) return fail(c, PM_ERR_INVALID, "pm_kick: pos/vel is NULL");
  if (!c->deposited || !c->have_response) return fail(c, PM_ERR_ORDER, "pm_kick needs pm_deposit and pm_nu_response first");
  if (c->power_set) return fail(c, PM_ERR_ORDER, "pm_kick after pm_set_power needs a new pm_deposit");
  if (a != c->a_response) return fail(c, PM_ERR_ORDER, "pm_kick at a different a than pm_nu_response");
  if (!isfinite(kick_factor)) return fail(c, PM_ERR_INVALID, "kick_factor must be finite");
  GridArgs g = grid_args(c);
  int rc = PM_OK;
  {
    Stage st(c, PM_ST_GREEN, 1);
    rc = c->fp64 ? green_f64(g, c->stream) : green_f32(g, c->stream);
  }
  c->deposit_grid_valid = false;
  // the row-order gather walks the deposit's sort: only for the same positions
  g.rows_ready = ((c->gather_rows == 1 && c->perm_valid) || (c->gather_rows == 2 && c->inv_valid)) &&
                 pos == c->dep_pos && g.fd_grad;
  // the fused gather walks the row sort of pm_deposit, absent on the unfused path
  const bool separate = !(c->p.flags & PM_FUSED_GATHER) || (c->p.flags & PM_UNFUSED_DEPOSIT);
  const int inv[3] = {kPassZInv, kPassYInv, kPassXInv};
  const int ist[3] = {PM_ST_FFT_Z_INV, PM_ST_FFT_Y_INV, PM_ST_FFT_X_INV};
  for (int i = 0; i < 2 && rc == PM_OK; ++i) {
    Stage st(c, ist[i], 1);
    rc = c->fp64 ? fft_pass_f64(g, inv[i], c->stream) : fft_pass_f32(g, inv[i], c->stream);
  }
  if (separate) {
    if (rc == PM_OK) {
      Stage st(c, ist[2], 1);
      rc = c->fp64 ? fft_pass_f64(g, inv[2], c->stream) : fft_pass_f32(g, inv[2], c->stream);
    }
    if (rc == PM_OK) {
      Stage st(c, PM_ST_INTERP, g.rows_ready && c->gather_rows == 2 ? 2 : 1);
      rc = c->fp64 ? interp_f64(g, pos, vel, kick_factor, acc_out, c->stream)
                   : interp_f32(g, pos, vel, kick_factor, acc_out, c->stream);
    }
  } else if (rc == PM_OK) {
    // the row sort of pm_deposit lists the particles of each row (same positions)
    Stage st(c, PM_ST_FFT_X_INV, 1);
    rc = c->fp64 ? xinv_interp_f64(g, pos, vel, kick_factor, acc_out, c->stream)
                 : xinv_interp_f32(g, pos, vel, kick_factor, acc_out, c->stream);
  }
  if (rc != PM_OK) return fail(c, rc, "pm_kick: unsupported grid");
  rc = cuda_check(c, cudaGetLastError(), "pm_kick launch");
  if (rc == PM_OK) c->have_kick = separate;   // force grids exist only on the separate path
  return rc;
}

int pm_drift(pm_ctx* c, void* pos, const void* vel, double drift_factor) {
  if (!c) return PM_ERR_INVALID;
  if (!pos || !vel) return fail(c, PM_ERR_INVALID, "pm_drift: pos/vel is NULL");
  if (!isfinite(drift_factor)) return fail(c, PM_ERR_INVALID, "pm_drift: drift_factor must be finite");
  GridArgs g = grid_args(c);
  {
    Stage st(c, PM_ST_DRIFT, 1);
    const int rc = c->fp64 ? drift_f64(g, pos, vel, drift_factor, c->stream)
                           : drift_f32(g, pos, vel, drift_factor, c->stream);
    if (rc != PM_OK) return fail(c, rc, "pm_drift failed");
  }
  // the particles moved: a sort of the old positions no longer describes them
  c->perm_valid = false;
  c->inv_valid = false;
  return cuda_check(c, cudaGetLastError(), "pm_drift launch");
}

int pm_history_set(pm_ctx* c, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist,
                   const double* sqrtPnu_prev) {
  if (!c) return PM_ERR_INVALID;
  if (n_hist < 0 || n_hist > c->p.n_hist_max) return fail(c, PM_ERR_INVALID, "pm_history_set: n_hist outside 0..n_hist_max");
  if (n_hist > 0 && (!a_hist || !sqrtPM_hist)) return fail(c, PM_ERR_INVALID, "pm_history_set: NULL history");
  for (int j = 0; j < n_hist; ++j) {
    if (!isfinite(a_hist[j]) || (j == 0 && a_hist[0] < c->a_init) || (j > 0 && !(a_hist[j] > a_hist[j - 1])))
      return fail(c, PM_ERR_RANGE, "pm_history_set: a_hist must be finite, >= a_init and strictly increasing");
  }
  int rc = PM_OK;
  if (n_hist > 0)
    rc = cuda_check(c, cudaMemcpyAsync(c->d_hist_own, sqrtPM_hist, (size_t)n_hist * c->nk * sizeof(double),
                                       cudaMemcpyDeviceToDevice, c->stream), "pm_history_set copy");
  if (rc == PM_OK && sqrtPnu_prev)
    rc = cuda_check(c, cudaMemcpyAsync(c->d_prev[0], sqrtPnu_prev, (size_t)c->nk * sizeof(double),
                                       cudaMemcpyDeviceToDevice, c->stream), "pm_history_set copy");
  if (rc != PM_OK) return rc;
  c->own_a.assign(a_hist ? a_hist : a_hist, a_hist ? a_hist + n_hist : a_hist);
  c->prev_cur = 0;
  c->have_prev = sqrtPnu_prev != nullptr;
  return PM_OK;
}

int pm_history_get(pm_ctx* c, double* a_hist, double* sqrtPM_hist, double* sqrtPnu_prev, int32_t* n_hist) {
  if (!c) return PM_ERR_INVALID;
  const int n = (int)c->own_a.size();
  if (n_hist) *n_hist = n;
  if (a_hist)
    for (int j = 0; j < n; ++j) a_hist[j] = c->own_a[j];
  int rc = PM_OK;
  if (sqrtPM_hist && n > 0)
    rc = cuda_check(c, cudaMemcpyAsync(sqrtPM_hist, c->d_hist_own, (size_t)n * c->nk * sizeof(double),
                                       cudaMemcpyDeviceToDevice, c->stream), "pm_history_get copy");
  if (rc == PM_OK && sqrtPnu_prev && c->have_prev)
    rc = cuda_check(c, cudaMemcpyAsync(sqrtPnu_prev, c->d_prev[c->prev_cur], (size_t)c->nk * sizeof(double),
                                       cudaMemcpyDeviceToDevice, c->stream), "pm_history_get copy");
  return rc;
}

int pm_step(pm_ctx* c, void* pos, void* vel, double a, double kick_factor, double drift_factor, void* acc_out) {
  if (!c) return PM_ERR_INVALID;
  if (!pos || !vel) return fail(c, PM_ERR_INVALID, "pm_step: pos/vel is NULL");
  if (!isfinite(drift_factor)) return fail(c, PM_ERR_INVALID, "pm_step: drift_factor must be finite");
  const int n = (int)c->own_a.size();
  if (n >= c->p.n_hist_max) return fail(c, PM_ERR_RANGE, "pm_step: the stored history is full (n_hist_max rows)");
  if (n > 0 && !(a > c->own_a.back())) return fail(c, PM_ERR_RANGE, "pm_step: a must exceed the last stored a");
  const double* ah = n > 0 ? c->own_a.data() : nullptr;
  const double* hist = n > 0 ? c->d_hist_own : nullptr;
  // (iii) history panels on the side stream, overlapping the deposit
  int rc = pm_nu_prepare(c, a, ah, hist, n);
  // (ii) deposit, P_cdm
  if (rc == PM_OK) rc = pm_deposit(c, pos);
  // (iii) response; its P_M^{1/2} row is written straight into the history
  const int nxt = 1 - c->prev_cur;
  if (rc == PM_OK)
    rc = pm_nu_response(c, a, ah, hist, n, c->have_prev ? c->d_prev[c->prev_cur] : nullptr, nullptr, c->d_prev[nxt],
                        c->d_hist_own + (size_t)n * c->nk);
  // (iv) delta_M, Poisson, forces, kick
  if (rc == PM_OK) rc = pm_kick(c, pos, vel, a, kick_factor, acc_out);
  if (rc != PM_OK) {
    join_prepared(c);
    return rc;
  }
  c->own_a.push_back(a);
  c->prev_cur = nxt;
  c->have_prev = true;
  // (ii) of the next step: the particles move on
  if (drift_factor != 0.0) rc = pm_drift(c, pos, vel, drift_factor);
  return rc;
}

int pm_check(pm_ctx* c) {
  if (!c) return PM_ERR_INVALID;
  int rc = cuda_check(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                      "status read");
  if (rc == PM_OK) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "pm_check sync");
  if (rc != PM_OK) return rc;
  const int st = *c->h_status;
  if (st != 0) {
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    return fail(c, st, st == PM_ERR_RANGE ? "device: particle offset outside [0,1) or non-finite position"
                                          : "device: error recorded by a kernel");
  }
  return PM_OK;
}

void pm_free(pm_ctx* c) {
  if (!c) return;
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  release(c);
  delete c;
}

const char* pm_last_error(const pm_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

double pm_kick_factor(const pm_ctx* c, double a0, double a1) {
  if (!c || !(a0 > 0) || !(a1 > 0) || !isfinite(a0) || !isfinite(a1)) return NAN;
  return integrate_u(log(a0), log(a1), [c](double u) { return 1.0 / hubble(c, exp(u)); });
}

double pm_drift_factor(const pm_ctx* c, double a0, double a1) {
  if (!c || !(a0 > 0) || !(a1 > 0) || !isfinite(a0) || !isfinite(a1)) return NAN;
  return integrate_u(log(a0), log(a1), [c](double u) {
    const double a = exp(u);
    return 1.0 / (a * a * hubble(c, a));
  });
}

double pm_hubble(const pm_params* p, double a) {
  if (!p || !(a > 0) || !isfinite(a) || !(p->h > 0)) return NAN;
  double ms[3], mtot = 0.0, onu = 0.0;
  int ns = 0;
  species_setup(*p, ms, ns, mtot, onu);
  if (!(p->flags & PM_RELATIVISTIC)) {
    const double om = p->omega_cdm + onu;
    return sqrt(om / (a * a * a) + (1.0 - om));
  }
  // species weights m_s / M_nu over the massive species
  double w[3] = {0, 0, 0}, m[3] = {0, 0, 0}, wsum = 0.0;
  int k = 0;
  for (int i = 0; i < ns; ++i) wsum += ms[i];
  for (int i = 0; i < ns; ++i)
    if (ms[i] > 0) {
      m[k] = ms[i];
      w[k] = ms[i] / wsum;
      ++k;
    }
  RelBackground B{};
  fill_background(*p, m, w, k, onu, n_massive_of(ms, ns, onu), B);
  return sqrt(rel_e2(a, B));
}

int pm_get_bins(pm_ctx* c, double* count, double* ksum, double* psum) {
  if (!c) return PM_ERR_INVALID;
  if (!c->deposited) return fail(c, PM_ERR_ORDER, "pm_get_bins before pm_deposit");
  std::vector<double> h(3 * (size_t)c->nk);
  int rc = cuda_check(c, cudaMemcpyAsync(h.data(), c->d_bins, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream), "bins read");
  if (rc == PM_OK) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "bins sync");
  if (rc != PM_OK) return rc;
  if (count) memcpy(count, h.data(), c->nk * sizeof(double));
  if (ksum) memcpy(ksum, h.data() + c->nk, c->nk * sizeof(double));
  if (psum) memcpy(psum, h.data() + 2 * c->nk, c->nk * sizeof(double));
  return PM_OK;
}

int pm_get_thresholds(const pm_ctx* c, int64_t* t) {
  if (!c || !t) return PM_ERR_INVALID;
  for (size_t i = 0; i < c->thr.size(); ++i) t[i] = c->thr[i];
  return PM_OK;
}

int pm_copy_field(pm_ctx* c, int32_t which, void* dst) {
  if (!c || !dst) return PM_ERR_INVALID;
  const int64_t n3 = (int64_t)c->n * c->n * c->n;
  const size_t real = c->fp64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  switch (which) {
    case PM_FIELD_DEPOSIT:
      if (!c->deposit_grid_valid)
        return fail(c, PM_ERR_ORDER, "deposit grid not kept (needs PM_KEEP_DEPOSIT or PM_UNFUSED_DEPOSIT, "
                                     "after pm_deposit and before pm_kick)");
      e = cudaMemcpyAsync(dst, c->g, (size_t)n3 * 8, cudaMemcpyDeviceToDevice, c->stream);
      break;
    case PM_FIELD_DELTA_K: {
      if (!c->deposited) return fail(c, PM_ERR_ORDER, "no spectrum before pm_deposit");
      GridArgs g = grid_args(c);
      const int rc = c->fp64 ? unpack_f64(g, dst, c->stream) : unpack_f32(g, dst, c->stream);
      if (rc != PM_OK) return fail(c, rc, "unpack failed");
      e = cudaGetLastError();
      break;
    }
    case PM_FIELD_ACC_X:
    case PM_FIELD_ACC_Y:
    case PM_FIELD_ACC_Z: {
      if (!c->have_kick)
        return fail(c, PM_ERR_ORDER, "no force grids (before pm_kick, or pm_kick ran with PM_FUSED_GATHER)");
      const int comp = which - PM_FIELD_ACC_X;
      GridArgs g = grid_args(c);
      if (g.fd_grad) {   // the stencil on the potential grid, as the gather applies it
        const int rc = c->fp64 ? fd_field_f64(g, comp, dst, c->stream) : fd_field_f32(g, comp, dst, c->stream);
        if (rc != PM_OK) return fail(c, rc, "force field failed");
        e = cudaGetLastError();
        break;
      }
      const char* src = reinterpret_cast<const char*>(c->g) + (size_t)comp * c->field_elems * c->cplx;
      e = cudaMemcpyAsync(dst, src, (size_t)n3 * real, cudaMemcpyDeviceToDevice, c->stream);
      break;
    }
    case PM_FIELD_PHI: {
      if (!c->have_kick || !grid_args(c).fd_grad)
        return fail(c, PM_ERR_ORDER, "no potential grid (before pm_kick, or the gradient ran in Fourier space)");
      e = cudaMemcpyAsync(dst, c->g, (size_t)n3 * real, cudaMemcpyDeviceToDevice, c->stream);
      break;
    }
    default:
      return fail(c, PM_ERR_INVALID, "unknown field");
  }
  return cuda_check(c, e, "pm_copy_field");
}

int pm_timing(pm_ctx* c, int32_t enable) {
  if (!c) return PM_ERR_INVALID;
  const int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "pm_timing sync");
  if (rc != PM_OK) return rc;
  drain_timing(c);
  for (int i = 0; i < PM_NSTAGES; ++i) {
    c->st_ms[i] = 0;
    c->st_launch[i] = 0;
    c->st_calls[i] = 0;
  }
  c->timing = enable != 0;
  return PM_OK;
}

int pm_get_timing(pm_ctx* c, double* ms, int64_t* launches, int64_t* calls) {
  if (!c) return PM_ERR_INVALID;
  const int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "pm_get_timing sync");
  if (rc != PM_OK) return rc;
  drain_timing(c);
  for (int i = 0; i < PM_NSTAGES; ++i) {
    if (ms) ms[i] = c->st_ms[i];
    if (launches) launches[i] = c->st_launch[i];
    if (calls) calls[i] = c->st_calls[i];
  }
  return PM_OK;
}

int64_t pm_device_bytes(const pm_ctx* c) { return c ? c->bytes : 0; }

// gather_rows 2 needs the inverse permutation and the sorted forces (4 + 16
// bytes a particle in FP32, 4 + 32 in FP64), allocated on first use.
static int ensure_rows_acc(pm_ctx* c) {
  int rc = PM_OK;
  if (!c->d_inv) rc = dalloc(c, (void**)&c->d_inv, (size_t)c->np * sizeof(int), "inverse row permutation");
  if (rc == PM_OK && !c->d_accs)
    rc = dalloc(c, &c->d_accs, (size_t)c->np * 4 * (c->fp64 ? sizeof(double) : sizeof(float)), "sorted forces");
  return rc;
}

int pm_autotune(pm_ctx* c, const void* pos, void* vel, double a, const double* a_hist, const double* sqrtPM_hist,
                int32_t n_hist, int32_t reps, int32_t* tuned) {
  if (!c) return PM_ERR_INVALID;
  if (!pos || !vel) return fail(c, PM_ERR_INVALID, "pm_autotune: pos/vel is NULL");
  if (reps < 1) return fail(c, PM_ERR_INVALID, "pm_autotune: reps must be >= 1");
  const bool was_timing = c->timing;
  // total ms of the given stages over `reps` kicks (kick factor 0: velocities unchanged)
  auto measure = [&](const int* stages, int n_stages, double* out) -> int {
    int rc = pm_timing(c, 1);
    for (int r = 0; r < reps && rc == PM_OK; ++r) {
      rc = pm_deposit(c, pos);
      if (rc == PM_OK) rc = pm_nu_response(c, a, a_hist, sqrtPM_hist, n_hist, nullptr, nullptr, nullptr, nullptr);
      if (rc == PM_OK) rc = pm_kick(c, pos, vel, a, 0.0, nullptr);
    }
    if (rc != PM_OK) return rc;
    double ms[PM_NSTAGES];
    rc = pm_get_timing(c, ms, nullptr, nullptr);
    double t = 0.0;
    for (int i = 0; i < n_stages; ++i) t += ms[stages[i]];
    *out = t;
    return rc;
  };
  static const int kStY[2] = {PM_ST_FFT_Y_FWD, PM_ST_FFT_Y_INV};
  static const int kStZ[2] = {PM_ST_FFT_Z_FWD, PM_ST_FFT_Z_INV};
  static const int kStP[2] = {PM_ST_DEPOSIT, PM_ST_INTERP};
  int rc = PM_OK;
  double t0 = 0.0, t1 = 0.0;
  rc = measure(kStY, 1, &t0);   // warm-up: attributes, tables
  // column tiles of the y passes, then of the z passes
  for (int pass = 0; pass < 2 && rc == PM_OK; ++pass) {
    int& knob = pass == 0 ? c->wide_y : c->wide_z;
    const int* st = pass == 0 ? kStY : kStZ;
    knob = 0;
    rc = measure(st, 2, &t0);
    if (rc != PM_OK) break;
    knob = 1;
    rc = measure(st, 2, &t1);
    if (rc != PM_OK) break;
    knob = t1 < t0 ? 1 : 0;
    if (pass == 1 && c->tma_z16) {   // TMA-staged z passes
      double t2 = 0.0;
      const int prev = knob;
      knob = 2;
      rc = measure(st, 2, &t2);
      if (rc != PM_OK) break;
      knob = t2 < (t1 < t0 ? t1 : t0) ? 2 : prev;
    }
  }
  // CTAs per SM of the particle kernels (row sort, gather + kick)
  if (rc == PM_OK) {
    const int cand[4] = {4, 8, 16, 32};
    double best = 1e300;
    int best_c = 16;
    for (int i = 0; i < 4 && rc == PM_OK; ++i) {
      c->part_cps = cand[i];
      double t = 0.0;
      rc = measure(kStP, 2, &t);
      if (t < best) {
        best = t;
        best_c = cand[i];
      }
    }
    c->part_cps = best_c;
  }
  // gather order: particle order, or the row order of the deposit's sort
  // (records + permutation; the default real-space gradient on the sorted path)
  if (rc == PM_OK && c->d_perm && !(c->p.flags & (PM_SPECTRAL_GRADIENT | PM_FUSED_GATHER | PM_TMA_COLUMNS))) {
    double t[3] = {0.0, 1e300, 1e300};
    c->gather_rows = 0;
    rc = measure(kStP, 2, &t[0]);
    if (rc == PM_OK) {
      c->gather_rows = 1;
      rc = measure(kStP, 2, &t[1]);
    }
    // the forces-by-slot form only where its 20 (FP32) or 36 (FP64) bytes a
    // particle can be had; otherwise it is left out of the comparison
    if (rc == PM_OK && ensure_rows_acc(c) == PM_OK) {
      c->gather_rows = 2;
      rc = measure(kStP, 2, &t[2]);
    }
    int best = 0;
    for (int k = 1; k < 3; ++k)
      if (t[k] < t[best]) best = k;
    c->gather_rows = rc == PM_OK ? best : 0;
  }
  const int rc2 = pm_timing(c, was_timing ? 1 : 0);
  if (rc != PM_OK) return rc;
  if (rc2 != PM_OK) return rc2;
  c->have_response = false;   // the tuning kicks used a response the caller did not ask for
  if (tuned) {
    tuned[0] = c->wide_y;
    tuned[1] = c->wide_z;
    tuned[2] = c->part_cps;
    tuned[3] = c->gather_rows;
  }
  return PM_OK;
}

int pm_set_tuning(pm_ctx* c, const int32_t* tuned) {
  if (!c || !tuned) return PM_ERR_INVALID;
  if (tuned[0] < -1 || tuned[0] > 1 || tuned[1] < -1 || tuned[1] > 2 || tuned[2] < 1 || tuned[2] > 64 ||
      tuned[3] < 0 || tuned[3] > 2)
    return fail(c, PM_ERR_INVALID,
                "pm_set_tuning: wide_y in -1..1, wide_z in -1..2, ctas_per_sm in 1..64, gather_rows 0..2");
  if (tuned[1] == 2 && !c->tma_z16)
    return fail(c, PM_ERR_UNSUPPORTED, "pm_set_tuning: wide_z = 2 needs a power-of-two grid of 256 or more");
  if (tuned[3] == 2) {
    const int rc = ensure_rows_acc(c);
    if (rc != PM_OK) return rc;
  }
  c->wide_y = tuned[0];
  c->wide_z = tuned[1];
  c->part_cps = tuned[2];
  c->gather_rows = tuned[3];
  return PM_OK;
}

// ---- CUDA graphs of whole kicks ----
struct GraphHolder {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int pm_graph_begin(void* stream) {
  const cudaError_t e = cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal);
  return e == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

int pm_graph_end(void* stream, pm_graph** out) {
  if (!out) return PM_ERR_INVALID;
  *out = nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g) != cudaSuccess || !g) return PM_ERR_CUDA;
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PM_ERR_CUDA;
  }
  GraphHolder* h = new (std::nothrow) GraphHolder;
  if (!h) {
    cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    return PM_ERR_ALLOC;
  }
  h->graph = g;
  h->exec = ex;
  *out = reinterpret_cast<pm_graph*>(h);
  return PM_OK;
}

int pm_graph_launch(pm_graph* g, void* stream) {
  if (!g) return PM_ERR_INVALID;
  GraphHolder* h = reinterpret_cast<GraphHolder*>(g);
  return cudaGraphLaunch(h->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

int64_t pm_graph_nodes(const pm_graph* g) {
  if (!g) return 0;
  size_t n = 0;
  cudaGraphGetNodes(reinterpret_cast<const GraphHolder*>(g)->graph, nullptr, &n);
  return (int64_t)n;
}

void pm_graph_free(pm_graph* g) {
  if (!g) return;
  GraphHolder* h = reinterpret_cast<GraphHolder*>(g);
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  delete h;
}

}  // extern "C"

// ---- batched kicks of many boxes of one grid size (batch.cu) ----
struct pm_batch {
  std::vector<pm_ctx*> ctx;
  cudaStream_t stream = nullptr;
  int n = 0, nk = 0, hist_stride = 1;
  std::vector<int> first;              // [kBpPasses][nbox + 1]
  std::vector<int> bin_chunks;
  BatchPlan plan;
  int* d_first = nullptr;
  int* d_counters = nullptr;
  BoxArgs* d_boxes = nullptr;
  double* d_hist_u = nullptr;
  // staging (pinned): [0] eager kicks (reused after its copy completed), [1] a
  // captured kick (kept as the captured graph reads it at every replay)
  BoxArgs* h_boxes[2] = {nullptr, nullptr};
  double* h_hist_u[2] = {nullptr, nullptr};
  cudaEvent_t ev_staged = nullptr;
  bool staged_pending = false;
  cudaStream_t side = nullptr;             // the response panels beside the grid passes
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
};

extern "C" {

int pm_batch_create(pm_ctx* const* ctxs, int32_t nbox, void* cuda_stream, pm_batch** out) {
  if (!out) return PM_ERR_INVALID;
  *out = nullptr;
  if (!ctxs || nbox < 1) return PM_ERR_INVALID;
  const pm_ctx* c0 = ctxs[0];
  if (!c0) return PM_ERR_INVALID;
  const uint32_t bad_flags = PM_SPECTRAL_GRADIENT | PM_FUSED_GATHER | PM_TMA_COLUMNS | PM_UNFUSED_DEPOSIT;
  for (int b = 0; b < nbox; ++b) {
    const pm_ctx* c = ctxs[b];
    if (!c) return PM_ERR_INVALID;
    if (c->fp64 || c->n != c0->n || c->nk != c0->nk) {
      fprintf(stderr, "pm_batch_create: boxes must be PM_FP32 with one grid size and bin count\n");
      return PM_ERR_UNSUPPORTED;
    }
    if ((c->p.flags & bad_flags) || !batch_supported(c->n) || c->nk > 1024) {
      fprintf(stderr, "pm_batch_create: grid %d or flags not supported by the batched form\n", c->n);
      return PM_ERR_UNSUPPORTED;
    }
  }
  pm_batch* B = new (std::nothrow) pm_batch;
  if (!B) return PM_ERR_ALLOC;
  B->ctx.assign(ctxs, ctxs + nbox);
  B->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  B->n = c0->n;
  B->nk = c0->nk;
  for (int b = 0; b < nbox; ++b) B->hist_stride = std::max(B->hist_stride, ctxs[b]->p.n_hist_max + 1);
  B->first.assign((size_t)kBpPasses * (nbox + 1), 0);
  B->bin_chunks.resize(nbox);
  for (int b = 0; b < nbox; ++b) {
    const pm_ctx* c = ctxs[b];
    const int64_t rows = (int64_t)c->n * c->n;
    int chunks = (int)((rows + 31) / 32);
    if (chunks > c->nblk_bins) chunks = c->nblk_bins;
    B->bin_chunks[b] = chunks;
    const int ns = (c->ns > 0 && c->f_nu > 0) ? c->ns : 0;
    int items[kBpPasses];
    batch_items(c->n, c->np, c->nk, ns, chunks, items);
    for (int p = 0; p < kBpPasses; ++p) B->first[(size_t)p * (nbox + 1) + b + 1] = items[p];
  }
  for (int p = 0; p < kBpPasses; ++p)
    for (int b = 0; b < nbox; ++b) B->first[(size_t)p * (nbox + 1) + b + 1] += B->first[(size_t)p * (nbox + 1) + b];
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMalloc((void**)&B->d_first, B->first.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_counters, kBpPasses * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_boxes, (size_t)nbox * sizeof(BoxArgs));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_hist_u, (size_t)nbox * B->hist_stride * sizeof(double));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMallocHost((void**)&B->h_boxes[k], (size_t)nbox * sizeof(BoxArgs));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_hist_u[k], (size_t)nbox * B->hist_stride * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaMemcpy(B->d_first, B->first.data(), B->first.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pm_batch_free(B);
    return PM_ERR_ALLOC;
  }
  B->plan.n = B->n;
  B->plan.nbox = nbox;
  B->plan.nk = B->nk;
  B->plan.sm_count = sms;
  B->plan.d_boxes = B->d_boxes;
  B->plan.d_first = B->d_first;
  B->plan.h_first = B->first.data();
  B->plan.d_counters = B->d_counters;
  *out = B;
  return PM_OK;
}

int pm_batch_kick(pm_batch* B, const void* const* pos, void* const* vel, const double* a, const double* kick_factor,
                  const double* const* a_hist, const double* const* sqrtPM_hist, const int32_t* n_hist) {
  if (!B) return PM_ERR_INVALID;
  const int nbox = (int)B->ctx.size();
  if (!pos || !vel || !a || !kick_factor) {
    B->err = "pm_batch_kick: NULL argument array";
    return PM_ERR_INVALID;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(B->stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  const int stage = cap == cudaStreamCaptureStatusNone ? 0 : 1;
  if (stage == 0 && B->staged_pending) {   // the previous eager kick's copies have read the staging buffers
    if (cudaEventSynchronize(B->ev_staged) != cudaSuccess) {
      cudaGetLastError();
      return PM_ERR_CUDA;
    }
    B->staged_pending = false;
  }
  BoxArgs* hb = B->h_boxes[stage];
  double* hh = B->h_hist_u[stage];
  bool any_hist = false;
  for (int b = 0; b < nbox; ++b) {
    pm_ctx* c = B->ctx[b];
    const int nh = n_hist ? n_hist[b] : 0;
    const double* ah = a_hist ? a_hist[b] : nullptr;
    const double* hist = sqrtPM_hist ? sqrtPM_hist[b] : nullptr;
    char buf[160];
    snprintf(buf, sizeof buf, "pm_batch_kick: box %d: ", b);
    if (!pos[b] || !vel[b]) return B->err = std::string(buf) + "pos/vel NULL", PM_ERR_INVALID;
    if (!(isfinite(a[b]) && a[b] >= c->a_init) || !isfinite(kick_factor[b]))
      return B->err = std::string(buf) + "a or kick factor out of range", PM_ERR_RANGE;
    if (nh < 0 || nh > c->p.n_hist_max || (nh > 0 && (!ah || !hist)))
      return B->err = std::string(buf) + "bad history", PM_ERR_INVALID;
    for (int j = 0; j < nh; ++j)
      if (!isfinite(ah[j]) || (j == 0 && ah[0] < c->a_init) || (j > 0 && !(ah[j] > ah[j - 1])) ||
          (j == nh - 1 && !(ah[j] < a[b])))
        return B->err = std::string(buf) + "a_hist must increase from a_init to below a", PM_ERR_RANGE;
    if (c->prep_pending) return B->err = std::string(buf) + "pm_nu_prepare pending", PM_ERR_ORDER;
    const double ue = log(a[b]);
    if (ue > c->stab_umax) {
      const int rc = build_s_table(c, ue + 1.0);
      if (rc != PM_OK) return B->err = c->err, rc;
    }
    if (c->power_set) {   // the lattice count / |k| sums back in place of pm_set_power's values
      const int rc = cuda_check(c, cudaMemcpyAsync(c->d_bins, c->d_bins_lattice, 2 * (size_t)c->nk * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, B->stream), "lattice bins restore");
      if (rc != PM_OK) return B->err = c->err, rc;
      c->power_set = false;
    }
    if (c->counts_dirty) {   // the batched count adds to zeros; its scan clears them again
      const int rc = cuda_check(c, cudaMemsetAsync(c->d_rowc, 0, ((size_t)c->n * c->n + 1) * sizeof(int), B->stream),
                                "row count clear");
      if (rc != PM_OK) return B->err = c->err, rc;
      c->counts_dirty = false;
    }
    for (int j = 0; j < nh; ++j) hh[(size_t)b * B->hist_stride + j] = log(ah[j]);
    any_hist = any_hist || nh > 0;
    BoxArgs& x = hb[b];
    x.g = grid_args(c);
    const double coeff = -1.5 * c->omega_m / (a[b] * c->kf * c->kf * (double)c->n * c->n * c->n);
    x.g.green_coeff = (float)coeff;
    x.nu = nu_args(c, a[b], hist, nh, nullptr, nullptr, nullptr, nullptr);
    x.nu.hist_u = B->d_hist_u + (size_t)b * B->hist_stride;
    x.pos = pos[b];
    x.vel = vel[b];
    x.kick = (float)kick_factor[b];
    x.bin_chunks = B->bin_chunks[b];
    x.thr = c->d_thr;
    x.inv_lr = c->bin_inv_lr;
    x.kf = c->kf;
    x.fac_umax = 0.5 * log((double)c->n2max);
    x.partials = c->d_partials;
    x.psum = c->d_bins + 2 * c->nk;
    c->green_coeff = coeff;
  }
  cudaError_t e = cudaMemcpyAsync(B->d_boxes, hb, (size_t)nbox * sizeof(BoxArgs), cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess && any_hist)
    e = cudaMemcpyAsync(B->d_hist_u, hh, (size_t)nbox * B->hist_stride * sizeof(double), cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess && stage == 0) {
    e = cudaEventRecord(B->ev_staged, B->stream);
    B->staged_pending = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_counters, 0, kBpPasses * sizeof(int), B->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    B->err = std::string("pm_batch_kick: ") + cudaGetErrorString(e);
    return PM_ERR_CUDA;
  }
  int rc = batch_kick(B->plan, B->stream, B->side, B->ev_fork, B->ev_join);
  if (rc != PM_OK) return B->err = "pm_batch_kick: unsupported grid", rc;
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    B->err = std::string("pm_batch_kick launch: ") + cudaGetErrorString(e);
    return PM_ERR_CUDA;
  }
  for (int b = 0; b < nbox; ++b) {   // each context now holds this kick's results
    pm_ctx* c = B->ctx[b];
    c->deposited = true;
    c->have_response = true;
    c->a_response = a[b];
    c->have_kick = true;
    c->deposit_grid_valid = false;
    c->perm_valid = c->d_perm != nullptr && grid_args(c).perm != nullptr;
    c->inv_valid = false;   // the batched sort writes no inverse permutation
    c->dep_pos = pos[b];
  }
  return PM_OK;
}

int64_t pm_batch_launches(const pm_batch* B) {
  if (!B) return 0;
  int64_t k = 0;
  const int nbox = (int)B->ctx.size();
  for (int p = 0; p < kBpPasses; ++p) k += B->first[(size_t)p * (nbox + 1) + nbox] > 0 ? 1 : 0;
  return k;
}

const char* pm_batch_last_error(const pm_batch* B) { return B ? B->err.c_str() : "null batch"; }

void pm_batch_free(pm_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->d_first) cudaFree(B->d_first);
  if (B->d_counters) cudaFree(B->d_counters);
  if (B->d_boxes) cudaFree(B->d_boxes);
  if (B->d_hist_u) cudaFree(B->d_hist_u);
  for (int k = 0; k < 2; ++k) {
    if (B->h_boxes[k]) cudaFreeHost(B->h_boxes[k]);
    if (B->h_hist_u[k]) cudaFreeHost(B->h_hist_u[k]);
  }
  if (B->side) cudaStreamSynchronize(B->side);
  if (B->ev_staged) cudaEventDestroy(B->ev_staged);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  if (B->side) cudaStreamDestroy(B->side);
  delete B;
}

}  // extern "C"
