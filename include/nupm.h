/*
 * nupm.h -- C ABI of the GB300 particle-mesh (PM) long-range kick with
 * Fourier-space massive neutrinos (Ali-Haimoud & Bird, arXiv:1209.0461).
 *
 * One kick = the paper's Sec. 4.3 steps (ii)-(iv) at one time step:
 *   pm_deposit      fixed-point CIC deposit of the CDM particles, density
 *                   contrast, forward 3-D FFT and the binned P_cdm(k)
 *                   (Sec. 4.3 (ii));
 *   pm_nu_response  the neutrino linear response per |k| bin, Eq. P-final with
 *                   the initial-condition term of Eq. deltaI-nu and the
 *                   single-iteration implicit solve of Sec. 4.3 (iii)/App. B;
 *   pm_kick         delta_nu(k) = (P_nu/P_cdm)^{1/2} delta_cdm(k) (Eq. phases),
 *                   delta_M = (1-f_nu) delta_cdm + f_nu delta_nu (Sec. 4.3 (iv)),
 *                   Poisson (Eq. Poisson), gradient, inverse FFTs, CIC
 *                   interpolation and u += acc * K.
 *
 * Units: lengths in Mpc/h, time in 1/H0 (H0 = 1), velocities u = a^2 dx/dt in
 * H0 Mpc/h (100 km/s); superconformal time s = int dtau/a (Sec. 3.2).
 *
 * Memory: every pointer argument says HOST or DEVICE.  The context owns its
 * grids and tables (allocated at pm_init on the current device); the caller
 * owns particles, velocities and the stored spectra.  All GPU work is issued
 * on the stream given to pm_init and is asynchronous with respect to the
 * host; host arrays passed in are consumed before the call returns.
 *
 * Errors: every int-returning call returns PM_OK (0) or a negative PM_ERR_*
 * code; pm_last_error() gives a message.  Nothing throws across the ABI.
 * Host-side argument checks are reported by the call itself; conditions that
 * only the GPU can see (an offset outside [0,1), a non-finite position, a
 * fixed-point overflow) are recorded in a device status word and reported by
 * pm_check(), which synchronises the stream.
 */
#ifndef NUPM_H
#define NUPM_H

#include <stdint.h>

#if defined(__GNUC__)
#define NUPM_API __attribute__((visibility("default")))
#else
#define NUPM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PM_OK               0
#define PM_ERR_INVALID     -1   /* bad argument (NULL, size, non-finite parameter) */
#define PM_ERR_RANGE       -2   /* value outside its domain (offset not in [0,1), a < a_init, ...) */
#define PM_ERR_OVERFLOW    -3   /* a cell of the fixed-point deposit passed 2^64 - 1 (more than 65535
                                   particles' full weight in one cell): reported by pm_check after the
                                   deposit, whose grid is then wrong */
#define PM_ERR_CUDA        -4   /* a CUDA runtime call failed */
#define PM_ERR_ALLOC       -5   /* device allocation failed */
#define PM_ERR_TIMEOUT     -6   /* a bounded device wait gave up (reserved) */
#define PM_ERR_ORDER       -7   /* calls out of order (kick before deposit/response at this a) */
#define PM_ERR_UNSUPPORTED -8   /* grid size / option not built */

/* ---- precision of the grids, FFTs, positions and velocities ---- */
#define PM_FP64 0   /* positions: double[3][npart] comoving [Mpc/h]; grids FP64;   */
                    /* velocities double[3][npart]                                 */
#define PM_FP32 1   /* positions: int32 words [6][npart]: rows 0-2 the grid cell   */
                    /* index (any integer, wrapped), rows 3-5 the FP32 offset in   */
                    /* [0,1) stored bit-for-bit; grids FP32; velocities float[3][n] */

/* ---- flags ---- */
#define PM_I_FIT       0x1u  /* use the App. C fitting formula (Eq. fit) for I(x) */
#define PM_DECONV_CIC  0x2u  /* divide the Green function by prod sinc^4 (CIC windows) */
#define PM_KEEP_DEPOSIT 0x4u /* also write the fixed-point deposit grid (PM_FIELD_DEPOSIT) */
#define PM_UNFUSED_DEPOSIT 0x8u /* global-atomic deposit + separate x pass (no particle sort) */
#define PM_FUSED_GATHER 0x20u /* inverse x transform fused with the CIC gather + kick in a
                                 sliding window (no force grids; comparison: one CTA/SM on a
                                 1024^3 grid, slower than the separate pass + gather) */
#define PM_TMA_COLUMNS 0x10u /* column FFT passes as persistent TMA-pipelined kernels (comparison;
                                 1 CTA/SM: slower than the default on a 1024^3 grid) */
#define PM_SPECTRAL_GRADIENT 0x40u /* apply the 4-point gradient as its Fourier multiplier
                                 -i D(k): three force spectra, three inverse transforms, the
                                 gather reads three force grids (comparison).  Default: one
                                 inverse transform of the potential, and the gather applies
                                 the same 4-point difference to the real potential grid
                                 (equal in exact arithmetic).  PM_FUSED_GATHER and
                                 PM_TMA_COLUMNS imply it. */

#define PM_RELATIVISTIC 0x80u /* Sec. 4.4 background in H(a): each massive species with the
                                 energy density of Eq. relativistic (relativistic Fermi-Dirac
                                 momenta, T_nu0 = 1.68e-4 eV), radiation (photons, Omega_gamma
                                 h^2 = 2.4728e-5, and the massless of three neutrino species),
                                 Lambda closing the universe at a = 1.  Default: matter +
                                 Lambda with Omega_nu as matter.  Poisson keeps Omega_M. */

#define PM_IC_MULTIPOLE 0x100u /* initial-condition term of Eq. P-final by Eq. deltaI-multipole
                                 with the l = 0, 1 moments of Sec. 4.1: the l = 1 part from its
                                 own momentum integral of j_1 (FP64 Gauss-Legendre panels),
                                 -P_nu,i^{1/2} a_i [theta/delta]_i (s - s_i) K(y), instead of the
                                 integrated-by-parts Eq. deltaI-nu (K = I for these moments; the
                                 two agree to the quadrature's accuracy).  Beyond
                                 y = k (s - s_i) T_nu0 / m = 256 (K < 1e-10) K = I is used. */

/*
 * Problem statement (Sec. 4.3-4.4, Table 1).  Omega_M = omega_cdm + omega_nu
 * (baryons folded into cdm), flat: Omega_Lambda = 1 - Omega_M.
 *   omega_nu < 0       -> derived as m_nu_total_eV / (93.14 eV h^2) (Sec. 2.1)
 *   n_species          number of massive species (0..3); 0 or m_nu_total 0 -> no neutrinos
 *   m_nu_eV[i]         species masses; all zero -> degenerate m_nu_total / n_species
 *   particle_mass      uniform CDM particle mass (it cancels in delta; must be > 0)
 *   a_init             a_i of Eq. deltaI-nu (start of the response integral)
 *   n_kbins            log-spaced |k| bins on [2 pi/L, sqrt(3) pi N/L]
 *   n_hist_max         capacity the caller's stored-spectrum table may reach
 *   iters              implicit-solve iterations (Sec. 4.3 (iii), App. B), >= 1
 *   quad_nodes         Gauss-Legendre nodes per panel of the response integral (4..16)
 */
typedef struct {
  int32_t ngrid;          /* N: grid points per side: a power of two in 16..1024, or 192
                             (radix-3 transforms; not with PM_TMA_COLUMNS / PM_FUSED_GATHER) */
  int64_t npart;          /* number of CDM particles */
  double box;             /* L [Mpc/h] */
  double particle_mass;
  double omega_cdm, omega_nu, h;
  double m_nu_total_eV;
  int32_t n_species;
  double m_nu_eV[3];
  double a_init;
  int32_t n_kbins;
  int32_t n_hist_max;
  int32_t precision;      /* PM_FP64 | PM_FP32 */
  uint32_t flags;
  int32_t iters;
  int32_t quad_nodes;
} pm_params;

typedef struct pm_ctx pm_ctx;   /* opaque */

/* Fill *p with defaults (iters 1, quad_nodes 8, precision PM_FP64, no flags). */
NUPM_API void pm_default_params(pm_params* p);

/*
 * Create a context on the current CUDA device.
 *   sqrtPnu_init           HOST double[n_species][n_kbins]: P_nu,i^{1/2}(k_b) at a_init
 *                          (Eq. deltaI-nu), or NULL for unperturbed neutrinos at a_init
 *   theta_over_delta_init  HOST double[n_species][n_kbins]: [theta_nu/delta_nu]_i(k_b)
 *                          in units of H0 (Eq. P-final), or NULL for 0
 *   cuda_stream            cudaStream_t to issue all work on (NULL = legacy default)
 *   out                    receives the context; NULL on failure
 * Allocates the grids: FP32 4 N^2 (N/2) complex float, FP64 the same in double.
 */
NUPM_API int pm_init(const pm_params* params, const double* sqrtPnu_init,
            const double* theta_over_delta_init, void* cuda_stream, pm_ctx** out);

/*
 * Steps a1-a3 (Sec. 4.3 (ii)): CIC deposit of `pos` (DEVICE, layout by
 * precision, see PM_FP64/PM_FP32), delta = rho/rho_bar - 1, forward real 3-D
 * FFT and the binned CDM power spectrum (kept in the context).
 * Offsets outside [0,1) or non-finite positions set PM_ERR_RANGE in the
 * device status (see pm_check); their particles are skipped.
 */
NUPM_API int pm_deposit(pm_ctx* ctx, const void* pos);

/*
 * Step a4 (Eq. P-final, Eq. deltaI-nu, Sec. 4.3 (iii), App. B) at scale factor a
 * for every |k| bin, in FP64 on the GPU.
 *   a_hist        HOST double[n_hist]: scale factors of the stored spectra,
 *                 strictly increasing, a_init <= a_hist[0], a_hist[n-1] < a
 *   sqrtPM_hist   DEVICE double[n_hist][n_kbins]: stored P_M^{1/2}(k_b, a_j)
 *   n_hist        0..n_hist_max (0: initial-condition term only)
 *   sqrtPnu_prev  DEVICE double[n_kbins]: P_nu^{1/2} of the previous step (the
 *                 first-iteration guess of Sec. 4.3 (iii)), or NULL for the
 *                 species-weighted initial value
 *   ratio_out, sqrtPnu_out, sqrtPM_out
 *                 DEVICE double[n_kbins] or NULL: R_b = P_nu^{1/2}/P_cdm^{1/2},
 *                 P_nu^{1/2}(k_b, a), P_M^{1/2} = (1-f_nu) P_cdm^{1/2} + f_nu P_nu^{1/2}
 *                 (the row the caller appends to its history).  Empty bins give 0.
 * Requires pm_deposit first.  PM_ERR_RANGE for a < a_init or a bad history.
 */
NUPM_API int pm_nu_response(pm_ctx* ctx, double a, const double* a_hist, const double* sqrtPM_hist,
                   int32_t n_hist, const double* sqrtPnu_prev, double* ratio_out,
                   double* sqrtPnu_out, double* sqrtPM_out);

/*
 * Optional: start the history part of the next pm_nu_response before the
 * deposit.  The integral of Eq. P-final is linear in the current node of
 * P_M^{1/2} (the only part that needs this step's P_cdm), so its panels over
 * the stored history depend on the bins' |k| and the history alone.  This
 * launches them on the context's own side stream (forked from the context's
 * stream, so it runs after everything enqueued so far) where they overlap
 * pm_deposit's passes; the next pm_nu_response joins them and computes only
 * the current node, R and the tables.  Arguments as pm_nu_response; the
 * response uses the prepared panels when it gets the same a, a_hist values,
 * n_hist and sqrtPM_hist pointer and no pm_set_power came between (else it
 * recomputes them); the history must not change in between.  The results are
 * bit-identical to pm_nu_response alone.  A second pm_nu_prepare before the
 * response is PM_ERR_ORDER.  Under stream capture the side stream joins the
 * capture and the next pm_nu_response (or pm_nu_response_mlp,
 * pm_response_features) rejoins it.  The paper has no counterpart (the split
 * restates its integral, Sec. 4.3 (iii)).
 */
NUPM_API int pm_nu_prepare(pm_ctx* ctx, double a, const double* a_hist, const double* sqrtPM_hist,
                           int32_t n_hist);

/*
 * Steps a5-a7 (Eq. phases, Sec. 4.3 (iv), Eq. Poisson): Green function with the
 * neutrino factor (1-f_nu) + f_nu R(|k|), 4-point finite-difference gradient,
 * inverse FFTs, CIC interpolation with the deposit's weights and
 * vel += acc * kick_factor.
 *   pos          DEVICE, the same particles as the last pm_deposit
 *   vel          DEVICE, updated in place (double or float [3][npart] by precision)
 *   a            must equal the a of the last pm_nu_response (else PM_ERR_ORDER)
 *   kick_factor  K = int dt = int da/(a H) over the kick (pm_kick_factor)
 *   acc_out      DEVICE [3][npart] (precision's float type) or NULL
 */
NUPM_API int pm_kick(pm_ctx* ctx, const void* pos, void* vel, double a, double kick_factor,
            void* acc_out);

/*
 * Sec. 4.3 step (ii), "evolve the CDM ... up to the next timestep": move the
 * particles by Delta x = u Delta s (u = a^2 dx/dt, ds = dt / a^2, Sec. 3.1),
 * drift_factor = Delta s = pm_drift_factor(a0, a1).  In place on DEVICE pos,
 * with DEVICE vel (layouts of pm_deposit / pm_kick).  Each step is a fixed
 * sequence of IEEE roundings (no fused multiply-add), so results are the same
 * on every GPU:
 *   PM_FP64  x' = x + (u * ds); x' += L if x' < 0; x' -= L if x' >= L; a sum
 *            that rounds onto L becomes 0
 *   PM_FP32  g = (float)(ds / cell size); d = u * g; o' = o + d; k = floor(o');
 *            o'' = o' - k (o'' = 1 becomes 0 with k + 1); cell = (cell + k) mod N
 * A particle with a non-finite result, or an FP32 offset outside [0,1) on
 * entry, is left unchanged and sets PM_ERR_RANGE in the device status.
 */
NUPM_API int pm_drift(pm_ctx* ctx, void* pos, const void* vel, double drift_factor);

/*
 * The stored history of Sec. 4.3 kept by the context (pm_step appends to it).
 *   pm_history_set  replace it: a_hist HOST double[n_hist] (as pm_nu_response),
 *                   sqrtPM_hist DEVICE double[n_hist][n_kbins] (copied,
 *                   stream-ordered), sqrtPnu_prev DEVICE double[n_kbins] or NULL
 *                   (the next step's first-iteration guess; NULL = initial value);
 *                   n_hist 0..n_hist_max
 *   pm_history_get  HOST a_hist[n] and n_hist, DEVICE sqrtPM_hist[n][n_kbins]
 *                   and sqrtPnu_prev[n_kbins] (any may be NULL; DEVICE copies
 *                   are stream-ordered; sqrtPnu_prev is left unchanged when the
 *                   context has none)
 */
NUPM_API int pm_history_set(pm_ctx* ctx, const double* a_hist, const double* sqrtPM_hist, int32_t n_hist,
                            const double* sqrtPnu_prev);
NUPM_API int pm_history_get(pm_ctx* ctx, double* a_hist, double* sqrtPM_hist, double* sqrtPnu_prev,
                            int32_t* n_hist);

/*
 * One time step of Sec. 4.3 with the particles at scale factor a: steps
 * (ii)-(iv) -- pm_deposit, the response of Eq. P-final over the context's
 * stored history with the last step's P_nu^{1/2} as the first-iteration guess
 * (its history panels overlapping the deposit, as pm_nu_prepare), pm_kick
 * with kick_factor -- then "store the total matter power spectrum": the row
 * P_M^{1/2}(k_b, a) is appended to the context's history on the device and
 * P_nu^{1/2}(k_b, a) kept as the next guess, and finally pm_drift by
 * drift_factor (Delta s to the next step; 0 = no drift, e.g. after the last
 * step).  a must exceed the history's last scale factor; PM_ERR_RANGE when the
 * history already holds n_hist_max rows.  A leapfrog takes kick_factor =
 * K(a_{j-1/2}, a_{j+1/2}) (half steps at both ends) and drift_factor =
 * Delta s(a_j, a_{j+1}).  acc_out as pm_kick.
 */
NUPM_API int pm_step(pm_ctx* ctx, void* pos, void* vel, double a, double kick_factor, double drift_factor,
                     void* acc_out);

/* Synchronise the stream and report the first device-side error recorded
 * since the previous pm_check (then clear it). */
NUPM_API int pm_check(pm_ctx* ctx);

NUPM_API void pm_free(pm_ctx* ctx);
NUPM_API const char* pm_last_error(const pm_ctx* ctx);

/* H(a) / H0 of the background a problem statement describes (matter + Lambda,
 * or with PM_RELATIVISTIC in p->flags the Sec. 4.4 background), host FP64,
 * without a context or a GPU; NaN for a <= 0 or a NULL p. */
NUPM_API double pm_hubble(const pm_params* p, double a);

/* K = int_{a0}^{a1} da / (a H(a)) and Delta s = int da / (a^3 H(a)) of the
 * context's background, host FP64 (16-point Gauss-Legendre on panels of
 * width <= 1/8 in ln a); NaN on error. */
NUPM_API double pm_kick_factor(const pm_ctx* ctx, double a0, double a1);
NUPM_API double pm_drift_factor(const pm_ctx* ctx, double a0, double a1);

/* ---- inspection (tests, checkpointing) ---- */

/* Binned CDM spectrum of the last pm_deposit, HOST double[n_kbins] each (any may
 * be NULL): mode count sum w, sum w |k|, sum w |delta_k|^2 (w = 1 on the kx = 0
 * and kx = N/2 planes, 2 elsewhere).  Synchronises the stream. */
NUPM_API int pm_get_bins(pm_ctx* ctx, double* count, double* ksum, double* psum);

/* Integer n^2 thresholds of the bins, HOST int64[n_kbins + 1]. */
NUPM_API int pm_get_thresholds(const pm_ctx* ctx, int64_t* thresholds);

/* Copy an internal field to DEVICE memory `dst` (stream-ordered):
 *   PM_FIELD_DEPOSIT   uint64[N][N][N] fixed-point deposit (valid after pm_deposit,
 *                      until pm_kick overwrites it; needs PM_KEEP_DEPOSIT or
 *                      PM_UNFUSED_DEPOSIT)
 *   PM_FIELD_DELTA_K   the forward spectrum, complex[N][N][N/2+1] unpacked
 *                      (numpy rfftn layout), valid after pm_deposit
 *   PM_FIELD_ACC_X/Y/Z the real acceleration grids [N][N][N], valid after pm_kick
 *                      without PM_FUSED_GATHER (by default computed on request
 *                      from the potential with the gather's 4-point stencil)
 *   PM_FIELD_PHI       the real potential grid [N][N][N] (Eq. Poisson with the
 *                      neutrino-corrected delta_M), valid after pm_kick with
 *                      the default real-space gradient
 * Element type is the precision's float type (complex = 2 of them). */
#define PM_FIELD_DEPOSIT 0
#define PM_FIELD_DELTA_K 1
#define PM_FIELD_ACC_X   2
#define PM_FIELD_ACC_Y   3
#define PM_FIELD_ACC_Z   4
#define PM_FIELD_PHI     5
NUPM_API int pm_copy_field(pm_ctx* ctx, int32_t which, void* dst);

/* ---- per-stage timing (CUDA events on the context's stream) ----
 * Stages of one kick, in launch order. */
#define PM_ST_DEPOSIT    0   /* particle row sort (or, unfused, memset + CIC scatter) */
#define PM_ST_FFT_X_FWD  1   /* CIC deposit into row tiles + forward x transform */
#define PM_ST_FFT_Y_FWD  2
#define PM_ST_FFT_Z_FWD  3
#define PM_ST_BINS       4   /* P_cdm bins + fixed-order reduction */
#define PM_ST_RESPONSE   5   /* neutrino response + Green table */
#define PM_ST_GREEN      6
#define PM_ST_FFT_Z_INV  7
#define PM_ST_FFT_Y_INV  8
#define PM_ST_FFT_X_INV  9   /* inverse x transform (+ CIC gather + kick with PM_FUSED_GATHER) */
#define PM_ST_INTERP    10   /* CIC gather + kick (not launched with PM_FUSED_GATHER) */
#define PM_ST_DRIFT     11   /* pm_drift (also inside pm_step) */
#define PM_NSTAGES      12
/* enable != 0: record an event pair around every stage from now on and
 * clear the totals; 0: stop recording. */
NUPM_API int pm_timing(pm_ctx* ctx, int32_t enable);
/* Synchronise, then return per-stage totals since pm_timing(ctx, 1): HOST
 * ms[PM_NSTAGES] (elapsed GPU time), launches[PM_NSTAGES] (kernel launches),
 * calls[PM_NSTAGES] (times the stage ran); any pointer may be NULL. */
NUPM_API int pm_get_timing(pm_ctx* ctx, double* ms, int64_t* launches, int64_t* calls);

/*
 * Binned power spectrum of a caller-owned half spectrum, allocating no device
 * memory.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc -- codes that reserve all device memory for their
 * own pool at start-up, or that must not allocate inside their time-step loop
 * (an allocation can synchronise the device or fail mid-run) -- but still
 * want the P(k) diagnostic.  Its scratch (per-block partial sums) is a
 * fixed file-scope device array of 1.8 MB, held by every device that loads
 * the library until the process exits.
 *   spec        DEVICE complex [N][N][N/2+1] (numpy rfftn layout; double2 for
 *               PM_FP64, float2 for PM_FP32), e.g. pm_copy_field(PM_FIELD_DELTA_K)
 *   ngrid       N, a power of two in [16, 1024]
 *   n_kbins     1..256 (more is rejected with PM_ERR_RANGE)
 *   count, ksum, psum   DEVICE double[n_kbins] or NULL: sum w, sum w |k|,
 *               sum w |delta_k|^2 with the bins and weights of pm_get_bins
 *   cuda_stream stream to issue the work on
 * spec, the outputs and the stream must belong to the current device (a
 * stream on another device is rejected with PM_ERR_INVALID).  Each call made
 * outside a stream capture looks up the scratch array's device address
 * (cudaGetSymbolAddress) with the device current; a call under capture uses
 * the address of the last uncaptured call on that device, so make a first
 * call before any stream capture.  All calls on a device share the scratch:
 * each call rewrites all of it that it reads, but calls that overlap on the
 * GPU (different streams, no ordering between them) race.
 */
NUPM_API int pm_bin_power_static(const void* spec, int32_t ngrid, double box, int32_t n_kbins,
                                 int32_t precision, double* count, double* ksum, double* psum,
                                 void* cuda_stream);

/* The FP64 fused multiply-add rate of the current device in TFLOP/s (2 flops
 * per FMA), HOST *tflops, measured with CUDA events on cuda_stream over one
 * launch of eight independent FMA chains per thread (16 x 8 x iters FMAs a
 * thread, a few waves of resident CTAs); synchronises the stream.  The
 * denominator of the FP64 path's compute roofline: its transforms and
 * stencils run on the FP64 FMA pipe.  The paper has no counterpart. */
NUPM_API int pm_measure_fp64_fma(int32_t iters, double* tflops, void* cuda_stream);

/* Bytes of device memory the context holds. */
NUPM_API int64_t pm_device_bytes(const pm_ctx* ctx);

/* ---- autotuner ----
 * Times, on `reps` kicks of this context with the given particles (kick
 * factor 0, so velocities are unchanged), each candidate of
 *   wide_y / wide_z   column tiles of the y / z FFT passes: 0 = 64-byte row
 *                     segments (8 FP32 columns), 1 = 128-byte segments;
 *                     wide_z also 2 = 128-byte segments staged in shared
 *                     memory by TMA, the next tile's copy overlapping the
 *                     current tile's transform (power-of-two grids of 256
 *                     and more)
 *   ctas_per_sm       CTAs per SM of the particle kernels (row sort, CIC
 *                     gather): 4, 8, 16, 32
 *   gather_rows       0 = the CIC gather walks the particles in storage
 *                     order, 1 = in the row order of pm_deposit's sort (a
 *                     warp per grid row, velocities updated through the
 *                     sort's permutation), 2 = the same row order writing
 *                     each force by sorted slot, then the velocities updated
 *                     in storage order through the inverse permutation
 *                     (for particles far from their storage order; 20 bytes
 *                     a particle in FP32, 36 in FP64, allocated on first
 *                     use and left out if that allocation fails); 1 and 2
 *                     are used when pm_kick gets the same position pointer
 *                     as the deposit and need the sorted deposit and the
 *                     real-space gradient
 * one knob at a time, keeps the fastest and writes HOST tuned[4] = {wide_y,
 * wide_z, ctas_per_sm, gather_rows} (may be NULL).  a, a_hist, sqrtPM_hist, n_hist: as
 * pm_nu_response (the tuning kicks need a response).  Results are bit-identical
 * across choices except for the order of atomic arrival, which no output
 * depends on.  The paper has no counterpart (it is a property of this GPU). */
NUPM_API int pm_autotune(pm_ctx* ctx, const void* pos, void* vel, double a, const double* a_hist,
                         const double* sqrtPM_hist, int32_t n_hist, int32_t reps, int32_t* tuned);
/* Set the four knobs directly, HOST tuned[4] (-1 = built-in choice for wide_y / wide_z).
 * PM_ERR_INVALID for a value out of range, PM_ERR_UNSUPPORTED for wide_z = 2
 * on a grid that does not offer it, PM_ERR_ALLOC when gather_rows = 2 cannot
 * allocate its buffers (the tuning is then unchanged). */
NUPM_API int pm_set_tuning(pm_ctx* ctx, const int32_t* tuned);

/* ---- CUDA graphs of whole kicks (batched form) ----
 * pm_graph_begin starts capturing `stream` (thread-local capture mode);
 * pm_deposit, pm_nu_response, pm_nu_response_mlp and pm_kick calls of
 * contexts whose stream is `stream` -- or a stream joined to the capture by
 * an event recorded on it -- are recorded instead of run; pm_graph_end ends
 * the capture and instantiates the graph.  Each pm_graph_launch then replays
 * every recorded kick (velocities updated in place each time).  Capture
 * rules: run each recorded call once uncaptured first (kernel attributes and
 * tables are set up then), keep pm_timing off, do not call pm_check or
 * pm_get_* inside the capture, and keep the history pointers and values alive
 * and unchanged while the graph is used.  The paper has no counterpart. */
typedef struct pm_graph pm_graph;
NUPM_API int pm_graph_begin(void* cuda_stream);
NUPM_API int pm_graph_end(void* cuda_stream, pm_graph** out);
NUPM_API int pm_graph_launch(pm_graph* graph, void* cuda_stream);
NUPM_API int64_t pm_graph_nodes(const pm_graph* graph);
NUPM_API void pm_graph_free(pm_graph* graph);

/* ---- batched kicks (the batched form) ----
 * Boxes of ONE grid size stepped together: each pass of the kick (row count,
 * row scan, row scatter, deposit + x, y, z, bin sums and their reduction,
 * response panels, finish, bin list, fac table, Green plane, Green + z
 * inverse, y inverse, x inverse, gather + kick) is one persistent kernel over
 * all boxes, whose CTAs take (box, item) pairs -- particle chunks, row or
 * column tiles, response panels -- from an atomic counter until the pass's
 * work is done (no CTA waits on another).  Each box keeps its own context
 * (its grids, cosmology, neutrino masses, initial conditions, bins); the
 * batch only lists them.  A kick is pm_batch_launches(batch) kernel launches
 * plus three copies/memsets whatever the number of boxes, so a CUDA graph of it
 * (pm_graph_begin on the batch's stream) holds O(passes) nodes.  The paper
 * has no counterpart (its code steps one box).
 *   ctxs        HOST array of nbox contexts made by pm_init: PM_FP32, one grid
 *               size N (16..256 power of two, or 192), one n_kbins (<= 1024),
 *               the default path (none of PM_SPECTRAL_GRADIENT, PM_FUSED_GATHER,
 *               PM_TMA_COLUMNS, PM_UNFUSED_DEPOSIT); PM_ERR_UNSUPPORTED else
 *   cuda_stream the stream every batched kick is issued on
 * pm_batch_kick: per box b (HOST arrays of nbox entries): DEVICE pos[b] and
 * vel[b] (layouts of pm_kick, vel updated in place), scale factor a[b], kick
 * factor kick_factor[b], HOST a_hist[b][n_hist[b]] and DEVICE
 * sqrtPM_hist[b][n_hist[b]][n_kbins] (as pm_nu_response; a_hist, sqrtPM_hist
 * and n_hist may be NULL for no history).  Each box gets the kick pm_deposit +
 * pm_nu_response + pm_kick would give it (the same device code; the bin sums
 * are added in another order, so results agree to rounding, not bit for bit),
 * and its context holds that kick's bins, response and fields afterwards.
 * The host argument checks are those of pm_nu_response (PM_ERR_RANGE /
 * PM_ERR_INVALID, message in pm_batch_last_error); a context with a pending
 * pm_nu_prepare is PM_ERR_ORDER.  Under stream capture the kick's per-box
 * arguments are staged in a buffer kept for the graph: capture one kick per
 * batch, after an uncaptured one.  Contexts must outlive the batch. */
typedef struct pm_batch pm_batch;
NUPM_API int pm_batch_create(pm_ctx* const* ctxs, int32_t nbox, void* cuda_stream, pm_batch** out);
NUPM_API int pm_batch_kick(pm_batch* batch, const void* const* pos, void* const* vel, const double* a,
                           const double* kick_factor, const double* const* a_hist,
                           const double* const* sqrtPM_hist, const int32_t* n_hist);
NUPM_API int64_t pm_batch_launches(const pm_batch* batch);
NUPM_API const char* pm_batch_last_error(const pm_batch* batch);
NUPM_API void pm_batch_free(pm_batch* batch);

/* ---- learned response surrogate ----
 * The paper has no learned part; this stands in for the response integral of
 * pm_nu_response (Eq. P-final with Eq. deltaI-nu), which stays the fallback
 * and the yardstick its error is measured against.  A 3-layer perceptron
 *   h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2), out = w3 . h2 + b3,
 *   xh = (x - mu) / sigma,  ln R = y_mu + y_sigma out,
 * width 128, BF16 weight matrices (W1, W2, w3), FP32 biases, FP32 accumulation,
 * maps the PM_MLP_FEATURES features of one k bin
 *   x = (ln k_b [h/Mpc], ln a, M_nu [eV], Omega_nu, c_0 .. c_7)
 * to ln R_b, R_b = P_nu^{1/2}(k_b, a) / P_cdm^{1/2}(k_b, a).  c_j (j < 8) are the
 * Chebyshev coefficients, c_j = (2/8) sum_m g(u_m) cos(j pi (m + 1/2) / 8), of
 *   g(u) = ln( P_M^{1/2}(k_b, a'(u)) / P_cdm^{1/2}(k_b, a) ),
 *   u_m = ln a_i + (t_m + 1)/2 (ln a - ln a_i), t_m = cos(pi (m + 1/2) / 8),
 * with P_M^{1/2} linear in ln a' between the stored history nodes, closed by
 * the node (a, P_cdm^{1/2}(k_b, a)) and constant back to a_i.
 * Flat FP32 parameter layout (pm_mlp_param_count values):
 *   W1 [128][n_in], b1 [128], W2 [128][128], b2 [128], w3 [128], b3 [1].
 * Arrays marked DEVICE are device pointers; the work is ordered on the stream
 * given at creation.  Errors: PM_ERR_INVALID (bad sizes, NULL pointers),
 * PM_ERR_ALLOC, PM_ERR_CUDA. */
#define PM_MLP_FEATURES 12
#define PM_MLP_WIDTH 128
typedef struct pm_mlp pm_mlp;
/* n_in in 1..16, width must be PM_MLP_WIDTH.  Parameters start at zero (set
 * them with pm_mlp_set_params); normalisation starts at mu = 0, sigma = 1. */
NUPM_API int pm_mlp_create(int32_t n_in, int32_t width, void* cuda_stream, pm_mlp** out);
NUPM_API void pm_mlp_free(pm_mlp* mlp);
NUPM_API int64_t pm_mlp_param_count(const pm_mlp* mlp);
/* HOST float[pm_mlp_param_count]: the FP32 master copy (BF16 weight copies are
 * rounded from it to nearest even); resets the Adam moments and step count.
 * Synchronises the stream. */
NUPM_API int pm_mlp_set_params(pm_mlp* mlp, const float* host_params);
NUPM_API int pm_mlp_get_params(const pm_mlp* mlp, float* host_params);
/* HOST mu[n_in], sigma[n_in] (> 0) and the output scale (y_sigma > 0). */
NUPM_API int pm_mlp_set_norm(pm_mlp* mlp, const float* mu, const float* sigma, float y_mu, float y_sigma);
/* DEVICE X float[n][n_in] raw features -> DEVICE y float[n] = ln R. */
NUPM_API int pm_mlp_forward(pm_mlp* mlp, const float* X, int64_t n, float* y);
/* Gradient of L = (1/n) sum_i (out_i - (y_i - y_mu)/y_sigma)^2 with respect to
 * the parameters (the forward pass uses the BF16 weights), summed over CTAs
 * in a fixed order.  DEVICE grad float[param_count] and loss float[1], either
 * may be NULL. */
NUPM_API int pm_mlp_grad(pm_mlp* mlp, const float* X, const float* y, int64_t n, float* grad, float* loss);
/* pm_mlp_grad, then one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning
 * rate lr > 0) on the FP32 master copy and the BF16 copies.  DEVICE loss may
 * be NULL (the loss before the step). */
NUPM_API int pm_mlp_train_step(pm_mlp* mlp, const float* X, const float* y, int64_t n, float lr, float* loss);
/* The surrogate's features of every bin of the context's current P_cdm bins
 * (after pm_deposit or pm_set_power) at scale factor a with the stored history
 * (same arguments and checks as pm_nu_response): DEVICE X float[n_kbins][12];
 * rows of empty bins are zero. */
NUPM_API int pm_response_features(pm_ctx* ctx, double a, const double* a_hist, const double* sqrtPM_hist,
                                  int32_t n_hist, float* X);
/* pm_nu_response with the surrogate in place of the integral: R_b = exp(ln R_b)
 * for non-empty bins (0 for empty ones), P_nu^{1/2} = R_b P_cdm^{1/2},
 * P_M^{1/2} = (1 - f_nu) P_cdm^{1/2} + f_nu P_nu^{1/2}; prepares pm_kick exactly
 * as pm_nu_response does.  Outputs as pm_nu_response (DEVICE, may be NULL).
 * Without massive neutrinos it behaves as pm_nu_response (R = 0). */
NUPM_API int pm_nu_response_mlp(pm_ctx* ctx, pm_mlp* mlp, double a, const double* a_hist,
                                const double* sqrtPM_hist, int32_t n_hist, double* ratio_out,
                                double* sqrtPnu_out, double* sqrtPM_out);
/* Replace the context's P_cdm bins with caller values (HOST double[n_kbins]:
 * count, ksum = count k_b [h/Mpc], psum in the units of pm_get_bins) so that
 * pm_nu_response / pm_response_features can run on chosen spectra (e.g. to
 * generate the surrogate's training set from the exact integral).  pm_kick
 * then needs a new pm_deposit (PM_ERR_ORDER otherwise).  The paper has no
 * counterpart. */
NUPM_API int pm_set_power(pm_ctx* ctx, const double* count, const double* ksum, const double* psum);

#ifdef __cplusplus
}
#endif
#endif /* NUPM_H */
