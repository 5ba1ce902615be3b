// Internal declarations shared by the host API and the kernel translation
// units of libnupm.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/nupm.h"

namespace nupm {

constexpr double kCOverH0 = 2997.92458;   // c / H0 [Mpc/h]
constexpr double kTnu0eV = 1.68e-4;       // T_nu,0 [eV], Sec. 2.1 (value as printed)
constexpr double kOmegaNuEv = 93.14;      // Omega_nu h^2 = sum m / 93.14 eV, Sec. 2.1
constexpr int kMaxQuad = 16;
constexpr int kMaxPanels = 320;           // history nodes + graded points + ends
constexpr int kNuChunks = 10;             // warps per (bin, species), 32 panels each

// Integer n^2 thresholds of the |k| bins: T_b = ceil((e_b L / 2 pi)^2), b = 0..nk,
// for edges e_b log-spaced on [2 pi / L, sqrt(3) pi N / L (1 + 1e-12)]; a mode is in
// bin b iff T_b <= n^2 < T_{b+1}.  Shared by the context and the allocation-free
// binning entry point so that both bin every mode alike.
inline void bin_thresholds(int ngrid, int nk, long long* t) {
  const double r = sqrt(3.0) * ngrid / 2.0 * (1.0 + 1e-12);
  for (int b = 0; b <= nk; ++b) t[b] = (long long)ceil(pow(r, 2.0 * b / nk));
}
inline double bin_log_ratio(int ngrid) { return log(sqrt(3.0) * ngrid / 2.0 * (1.0 + 1e-12)); }

// ---- Sec. 4.4 background (PM_RELATIVISTIC) ----
// Radiation today: photons at T_cmb = 2.7255 K (Omega_gamma h^2 = 2.4728e-5)
// and each massless neutrino species (7/8)(4/11)^{4/3} of that; of three
// neutrino species, those without a mass are massless.
constexpr double kOmegaGammaH2 = 2.4728e-5;
constexpr int kNuSpeciesTotal = 3;
inline double nu_to_gamma() { return 7.0 / 8.0 * pow(4.0 / 11.0, 4.0 / 3.0); }
// R(y) = rho_nu / rho_nu,NR of one massive species (Eq. relativistic), y = m a / T_nu0,
// tabulated as ln R and d ln R / d ln y on t = ln y = kRelT0 + i kRelH (cubic
// Hermite in t); beyond the table the ultra- and non-relativistic series.
constexpr double kRelT0 = -9.210340371976182;    // ln 1e-4
constexpr double kRelH = 1.0 / 256.0;
constexpr int kRelN = 5896;                       // up to ln y = kRelT0 + (kRelN - 1) kRelH > ln 1e6
constexpr double kRelZeta3 = 1.2020569031595942, kRelZeta5 = 1.0369277551433699, kRelPi = 3.141592653589793;
// y R -> 7 pi^4 / (180 zeta 3) (1 + 5 y^2 / (7 pi^2)) as y -> 0; R - 1 -> 15 zeta(5) / (2 zeta(3) y^2) as y -> inf
constexpr double kRelUR = 7.0 * kRelPi * kRelPi * kRelPi * kRelPi / (180.0 * kRelZeta3);
constexpr double kRelUR2 = 5.0 / (7.0 * kRelPi * kRelPi);
constexpr double kRelNR = 15.0 * kRelZeta5 / (2.0 * kRelZeta3);
__host__ __device__ inline double nu_rho_ratio(double y, const double* tab) {
  const double t = log(y);
  const double u = (t - kRelT0) * (1.0 / kRelH);
  if (u < 0.0) return kRelUR / y * (1.0 + kRelUR2 * y * y);
  if (u >= (double)(kRelN - 1)) return 1.0 + kRelNR / (y * y);
  const int i = (int)u;
  const double f = u - i;
  const double y0 = tab[2 * i], d0 = tab[2 * i + 1] * kRelH, y1 = tab[2 * i + 2], d1 = tab[2 * i + 3] * kRelH;
  const double f2 = f * f, f3 = f2 * f;
  return exp((2 * f3 - 3 * f2 + 1) * y0 + (f3 - 2 * f2 + f) * d0 + (-2 * f3 + 3 * f2) * y1 + (f3 - f2) * d1);
}
// (H / H0)^2 of the Sec. 4.4 background: CDM a^-3, radiation a^-4, Lambda, and
// each massive species Omega_nu,s R(y1_s a) a^-3 (y1_s = m_s / T_nu0).
struct RelBackground {
  double om_cdm, om_r, om_lam;
  int ns;
  double om_nu[3], y1[3];
  const double* tab;
};
__host__ __device__ inline double rel_e2(double a, const RelBackground& B) {
  const double a3 = a * a * a;
  double e = B.om_cdm / a3 + B.om_r / (a3 * a) + B.om_lam;
  for (int s = 0; s < B.ns; ++s) e += B.om_nu[s] * nu_rho_ratio(B.y1[s] * a, B.tab) / a3;
  return e;
}

// I(x) on [kIX0, kIX0 + kISeg kIH) as kISeg Chebyshev pieces of kICoef terms,
// built once per context on the device from the exact I (launch_I_table).
constexpr double kIX0 = 0.5, kIH = 0.25;
constexpr int kISeg = 94, kICoef = 12;
void launch_I_table(double* coef, cudaStream_t s);

// Device inputs of the response kernels (one struct, passed by value).
struct NuArgs {
  int nk, ns, n_hist, quad, iters, use_fit, ngrid;
  double a, ue, ui, s_end;        // a, ln a, ln a_i, s(a) - s(a_i)
  double omega_m, omega_l, f_nu, a_init, box;
  double kappa_scale[3];          // c/H0 * T_nu0 / m_s (x = kappa_scale k (s - s'))
  double w_species[3];            // Omega_nu,s / Omega_nu
  const double* bins;             // [3][nk] count, ksum, psum
  const double* hist_u;           // [n_hist] ln a_j
  const double* hist;             // [n_hist][nk] P_M^{1/2}
  const double* prev;             // [nk] or nullptr
  const double* pnu_init;         // [ns][nk]
  const double* theta_init;       // [ns][nk]
  const double* stab;             // s-table: [n_stab][2] (s, ds/du) on a uniform u grid
  int n_stab;
  double stab_u0, stab_inv_h, stab_h;
  const double* gl;               // [2][quad] nodes, weights on [-1, 1]
  const double* icheb;            // [kISeg][kICoef] Chebyshev pieces of I(x)
  double* parts;                  // [ns][nk][kNuChunks][3] IC, J_hist, W_cur per panel chunk
  int nchunks;                    // chunks in use (<= kNuChunks), from a bound on the panel count
  double* rlist;                  // [2 nk + 1]: ln k_b and R_b of the non-empty bins, then their count
  double* R;                      // [nk]
  double* pnu;                    // [nk]
  double* pm;                     // [nk]
  double* R_user;                 // optional copies
  double* pnu_user;
  double* pm_user;
  int ic_multipole;               // 1: initial-condition term by Eq. deltaI-multipole (j_1 integral)
  int rel;                        // 1: H(a) of the Sec. 4.4 background (bg), else matter + Lambda
  RelBackground bg;
};

void launch_nu_response(const NuArgs& a, cudaStream_t s);
// the two halves of launch_nu_response: the history panels (they read the
// bins' |k| only, not P_cdm) and the current node, R and the bin list
void launch_nu_panels(const NuArgs& a, cudaStream_t s);
void launch_nu_finish(const NuArgs& a, cudaStream_t s);
// Surrogate: features [nk][12] of the bins and history in a (FP64 -> float),
// and the finish from the surrogate's ln R (R, P_nu, P_M, rlist).
void launch_nu_features(const NuArgs& a, double m_nu, double omega_nu, float* X, cudaStream_t s);
void launch_nu_from_lnR(const NuArgs& a, const float* lnR, cudaStream_t s);
// Surrogate network (mlp.cu): input count, and the forward pass on a given stream.
int mlp_inputs(const pm_mlp* m);
int mlp_forward_on(pm_mlp* m, const float* X, int64_t n, float* y, cudaStream_t s);
// fac(u) = (1 - f) + f R(k), ln k = ln kf + u, on kFacTable points of u in [0, umax]
// (u = ln sqrt(n^2)); the FP32 inverse z pass interpolates it linearly in u.
constexpr int kFacTable = 2048;
void launch_fac_table(float* fac, double umax, double kf, double f_nu, const double* rlist, int nk,
                      cudaStream_t s);
// Green table G(n^2), n^2 = 0..n2max, precision T; coeff = -1.5 Om / (a kf^2 N^3);
// rlist from the response (compacted non-empty bins)
void launch_green_table(bool fp64, void* gtab, long long n2max, double kf, double coeff,
                        double f_nu, const double* rlist, int nk, cudaStream_t s);

// FFT passes in launch order of one kick
constexpr int kPassXFwd = 0, kPassYFwd = 1, kPassZFwd = 2, kPassZInv = 3, kPassYInv = 4, kPassXInv = 5;

// precision-dispatched grid launchers (grid_f32.cu / grid_f64.cu)
struct GridArgs {
  int n;
  int64_t np;
  double box, delta, scale;       // scale = N^3 / (Np 2^48)
  void* spec;                     // packed spectrum [N][N][M]
  void* g;                        // 3 packed fields (deposit grid aliases the first two)
  int64_t field_elems;            // N*N*M complex elements per field
  const void* tw_n;               // W_N^m, m < N
  const void* tw_m;               // W_M^m, m < M
  int* status;
  const void* gtab;               // Green table G(n^2), grid precision
  const void* dtab;               // 4-point gradient multiplier per index
  const void* wtab;               // 1/sinc^4 per index, or nullptr (no deconvolution)
  void* plane0;                   // [N][N] complex: Green-multiplied packed column x2 = 0
  int* row_count;                  // [N^2 + 1] particles per row (sort)
  int* row_start;                  // [N^2 + 1] exclusive prefix of row_count
  int* row_cursor;                 // [N^2 + 1]
  int* scan_tot;                   // [2 * 1024] block totals of the scan
  int* perm;                       // [npart] particle indices sorted by row (fused gather only, else null)
  int* inv;                        // [npart] each particle's sorted slot, -1 if skipped (gather_rows 2, else null)
  void* accs;                      // [npart][4] forces in sorted order (gather_rows 2)
  unsigned long long* rec;         // [npart] packed particle records sorted by row
  const CUtensorMap* tmap_spec_y;  // TMA maps of the column passes (nullptr: plain kernels)
  const CUtensorMap* tmap_spec_z;
  const CUtensorMap* tmap_g_y;
  const CUtensorMap* tmap_bins = nullptr; // FP32 spectrum as [rows][32][E] 8-byte elements, 128-byte swizzle
  const CUtensorMap* tmap_z16 = nullptr;  // spectrum along z, 128-byte segments (wide_z = 2), or nullptr
  int sm_count;
  const float* fac;               // FP32 path: fac table (kFacTable points)
  float fac_inv_du;               // 1 / table spacing in u = ln sqrt(n^2)
  float green_coeff;              // -1.5 Omega_M / (a kf^2 N^3)
  // tuning (pm_autotune): wide (1) or narrow (0) column tiles of the y and z
  // passes, 2 = TMA-staged wide z passes, -1 = the built-in choice; CTAs per
  // SM of the particle kernels
  int wide_y = -1, wide_z = -1;
  int part_ctas_per_sm = 16;
  // gradient: false = -i D(k) in Fourier space (three inverse transforms of
  // force spectra); true = the 4-point stencil on the real potential grid,
  // applied by the gather (one inverse transform)
  bool fd_grad = false;
  // tuning: 1 = gather in the row order of the deposit's sort (records +
  // perm), 2 = the same order writing forces by sorted slot, then the
  // velocity update in particle order through inv; used when rows_ready (same
  // positions as the deposit, perm or inv written)
  int gather_rows = 0;
  bool rows_ready = false;
  // FP32 bin power sums inside the TMA-staged forward z pass (wide_z = 2,
  // n_kbins <= 256): the z pass writes one partial row per CTA, the bins step
  // adds the packed x2 = 0 column and reduces
  bool bins_in_z = false;
  const int* bin_thr = nullptr;
  float bin_inv_lr = 0;
  int bin_nk = 0;
  double* bin_partials = nullptr;
};
#define NUPM_DECLARE_GRID(SFX)                                                              \
  int deposit##SFX(const GridArgs& g, const void* pos, cudaStream_t s);                     \
  int row_sort##SFX(const GridArgs& g, const void* pos, cudaStream_t s);                    \
  int deposit_fft_x##SFX(const GridArgs& g, const void* pos, bool keep, cudaStream_t s);    \
  int fft_pass##SFX(const GridArgs& g, int pass, cudaStream_t s);                           \
  int bins##SFX(const GridArgs& g, bool lattice, int nk, const int* thr, float inv_lr,       \
                double kf, double* partials, int nblk, double* out, cudaStream_t s);        \
  int green##SFX(const GridArgs& g, cudaStream_t s);                                        \
  int interp##SFX(const GridArgs& g, const void* pos, void* vel, double kick, void* acc_out, \
                  cudaStream_t s);                                                          \
  int xinv_interp##SFX(const GridArgs& g, const void* pos, void* vel, double kick,          \
                       void* acc_out, cudaStream_t s);                                      \
  int unpack##SFX(const GridArgs& g, void* dst, cudaStream_t s);                            \
  int drift##SFX(const GridArgs& g, void* pos, const void* vel, double ds, cudaStream_t s);   \
  int fd_field##SFX(const GridArgs& g, int comp, void* dst, cudaStream_t s);
NUPM_DECLARE_GRID(_f32)
NUPM_DECLARE_GRID(_f64)
#undef NUPM_DECLARE_GRID

// ---- batched kicks of boxes of one grid size (batch.cu) ----
// One box of a batched kick (device copy, rewritten at every kick).
struct BoxArgs {
  GridArgs g;             // the box context's grids, tables, sort buffers and scalars
  NuArgs nu;              // its response arguments at this kick
  const void* pos;
  void* vel;
  float kick;
  int bin_chunks;         // rows of bin partial sums (row chunks of the spectrum)
  const int* thr;         // bin thresholds (int32, nk + 1)
  float inv_lr;
  double kf, fac_umax;    // 2 pi / L; ln sqrt(n^2_max) of the fac table
  double* partials;       // [bin_chunks][nk]
  double* psum;           // the box's sum w |delta|^2 per bin
};
enum BatchPass {
  kBpCount, kBpScan, kBpScatter, kBpDeposit, kBpY, kBpZ, kBpBins, kBpBinReduce, kBpPanels, kBpFinish, kBpRlist,
  kBpFac, kBpPlane0, kBpZInv, kBpYInv, kBpXInv, kBpGather, kBpPasses
};
struct BatchPlan {
  int n = 0, nbox = 0, nk = 0, sm_count = 0;
  BoxArgs* d_boxes = nullptr;
  int* d_first = nullptr;             // [kBpPasses][nbox + 1] first item of each box, then the total
  const int* h_first = nullptr;       // host copy
  int* d_counters = nullptr;          // [kBpPasses] work-queue counters, zeroed before each kick
};
// Items of each pass for one box (grid n, np particles, nk bins, ns response
// species, bin_chunks partials rows); the grid sizes the batch supports.
void batch_items(int n, int64_t np, int nk, int ns, int bin_chunks, int* items);
bool batch_supported(int n);
// The kick's passes on stream s; the response panels on `side`, forked after
// the staging copies (ev_fork) and joined before the finish (ev_join).
int batch_kick(const BatchPlan& p, cudaStream_t s, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join);

// out[i] = sum over blocks of partials[blk][i], i < len, in a fixed order
// (grid ceil(len / 32), 1024 threads).
__global__ void k_bin_reduce(const double* __restrict__ partials, int nblk, int len,
                             double* __restrict__ out);


}  // namespace nupm
