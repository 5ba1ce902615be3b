// Launchers of the grid kernels for one precision.  Included by grid_f32.cu
// and grid_f64.cu with NUPM_T set to float / double (one translation unit per
// precision so the two compile in parallel).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "grid_kernels.cuh"
#include "nupm_internal.h"
#include "sort.cuh"
#include "fft_tma.cuh"

namespace nupm {
namespace {

using T = NUPM_T;
using C = cx<T>;
constexpr int kSMs = 152;

// Shared memory of the Green z pass: exchange buffer, fac table (FP32) and
// the per-thread Green factors.
template <int N, class CC>
constexpr size_t green_smem() {
  return (size_t)CC::SMEM_WORDS * sizeof(C) + (sizeof(T) == 4 ? kFacTable * sizeof(float) : 0) +
         (size_t)CC::E * CC::THREADS * sizeof(T);
}
template <class CC>
constexpr size_t col_smem() {
  return (size_t)CC::SMEM_WORDS * sizeof(C);
}

// Opt the FFT kernels of size N into their dynamic shared memory (once per
// process; every kernel of this size gets its attribute on first use).
template <int N, class CC>
void col_attrs() {
  cudaFuncSetAttribute(k_fft_col<T, N, -1, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem<CC>());
  cudaFuncSetAttribute(k_fft_z_inv_green<T, N, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)green_smem<N, CC>());
  cudaFuncSetAttribute(k_fft_z_inv_green<T, N, CC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)green_smem<N, CC>());
  cudaFuncSetAttribute(k_fft_col<T, N, +1, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem<CC>());
  cudaFuncSetAttribute(k_fft_y_inv_grad<T, N, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)col_smem<CC>());
}
template <int N>
void ensure_attrs() {
  using RC = RowCfg<T, N>;
  static bool done = false;
  if (done) return;
  const int row_smem = (int)((size_t)RC::ROWS * RC::ROW_WORDS * sizeof(C));
  cudaFuncSetAttribute(k_fft_x_fwd<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, row_smem);
  cudaFuncSetAttribute(k_fft_x_inv<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, row_smem);
  col_attrs<N, ColNarrow<T, N>>();
  col_attrs<N, ColWide<T, N>>();
  done = true;
}

// Column passes with tile config CC: forward y / z, Green z, gradient y.
template <int N, class CC>
void col_pass(const GridArgs& g, int pass, cudaStream_t s) {
  constexpr int M = N / 2;
  const dim3 grid(M / CC::W, N, 1);
  const C* twn = reinterpret_cast<const C*>(g.tw_n);
  C* spec = reinterpret_cast<C*>(g.spec);
  C* f = reinterpret_cast<C*>(g.g);
  const int64_t fe = g.field_elems;
  switch (pass) {
    case kPassYFwd:
      k_fft_col<T, N, -1, CC><<<grid, CC::THREADS, col_smem<CC>(), s>>>(spec, (int64_t)N * M, (int64_t)M, 0, twn);
      break;
    case kPassZFwd:
      k_fft_col<T, N, -1, CC><<<grid, CC::THREADS, col_smem<CC>(), s>>>(spec, (int64_t)M, (int64_t)N * M, 0, twn);
      break;
    case kPassZInv:   // Green + z: spectrum -> g0 (phi), g2 (d/dz phi); real-space gradient: g0 only
      if (g.fd_grad) {
        k_fft_z_inv_green<T, N, CC, 1><<<grid, CC::THREADS, green_smem<N, CC>(), s>>>(
            spec, f, f + 2 * fe, reinterpret_cast<const C*>(g.plane0), reinterpret_cast<const T*>(g.gtab),
            reinterpret_cast<const T*>(g.dtab), reinterpret_cast<const T*>(g.wtab), twn, g.fac, g.fac_inv_du,
            g.green_coeff);
        break;
      }
      k_fft_z_inv_green<T, N, CC><<<grid, CC::THREADS, green_smem<N, CC>(), s>>>(
          spec, f, f + 2 * fe, reinterpret_cast<const C*>(g.plane0), reinterpret_cast<const T*>(g.gtab),
          reinterpret_cast<const T*>(g.dtab), reinterpret_cast<const T*>(g.wtab), twn, g.fac, g.fac_inv_du,
          g.green_coeff);
      break;
    case kPassYInv:   // y with the y gradient: g0 -> g1 (d/dy), g0 -> g0, g2 -> g2
      if (g.fd_grad) {   // the potential alone, in place
        k_fft_col<T, N, +1, CC><<<grid, CC::THREADS, col_smem<CC>(), s>>>(f, (int64_t)N * M, (int64_t)M, 0, twn);
        break;
      }
      k_fft_y_inv_grad<T, N, CC><<<grid, CC::THREADS, col_smem<CC>(), s>>>(
          f, f + fe, f + 2 * fe, reinterpret_cast<const T*>(g.dtab), twn);
      break;
  }
}

// TMA-pipelined column pass of size N.
template <int N, int MODE>
void col_tma_n(const GridArgs& g, const CUtensorMap* map, cudaStream_t s) {
  using Cfg = ColTmaCfg<T, N>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_col_tma<T, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    attr = true;
  }
  ColTmaArgs<T> a;
  a.spec = reinterpret_cast<C*>(g.spec);
  a.g = reinterpret_cast<C*>(g.g);
  a.field_elems = g.field_elems;
  a.tw = reinterpret_cast<const C*>(g.tw_n);
  a.plane0 = reinterpret_cast<const C*>(g.plane0);
  a.dtab = reinterpret_cast<const T*>(g.dtab);
  a.wtab = reinterpret_cast<const T*>(g.wtab);
  a.gtab = reinterpret_cast<const T*>(g.gtab);
  a.fac = g.fac;
  a.fac_inv_du = g.fac_inv_du;
  a.coeff = g.green_coeff;
  a.status = g.status;
  const int tiles = Cfg::TILES_PER_ROW * N;
  const int items = MODE == kColInvYGrad ? 2 * tiles : tiles;
  const int grid = items < g.sm_count ? items : g.sm_count;
  k_col_tma<T, N, MODE><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*map, a);
}

// The packed x2 = 0 column's bins after a forward z pass that summed the
// rest (FP32 grids of 256, 512 or 1024 points; false otherwise).  A template,
// so that the FP64 unit does not instantiate the FP32 kernels.
template <typename U>
bool bins_plane0(const GridArgs& g, int nk, const int* thr, float inv_lr, double* partials, int zgrid,
                 int nplane, cudaStream_t s) {
  if constexpr (sizeof(U) == 4) {
    const cx<float>* spec = reinterpret_cast<const cx<float>*>(g.spec);
    const size_t sh = (size_t)kPlaneBinWarps * nk * sizeof(float2);
    switch (g.n) {
      case 256: k_bin_plane0<256><<<nplane, kPlaneBinWarps * 32, sh, s>>>(spec, nk, thr, inv_lr, partials, zgrid); return true;
      case 512: k_bin_plane0<512><<<nplane, kPlaneBinWarps * 32, sh, s>>>(spec, nk, thr, inv_lr, partials, zgrid); return true;
      case 1024: k_bin_plane0<1024><<<nplane, kPlaneBinWarps * 32, sh, s>>>(spec, nk, thr, inv_lr, partials, zgrid); return true;
      default: return false;
    }
  }
  return false;
}

// Persistent grid of the TMA-staged forward z pass (one CTA per SM, at most
// one per tile): the number of partial rows its fused bin sums write.
static inline int z_fwd_grid(const GridArgs& g) {
  const int items = (g.n / 2 / ColTmaZCfg<float, 1024>::W) * g.n;
  return items < g.sm_count ? items : g.sm_count;
}

// TMA-staged z pass of size N with 128-byte segments (one resident CTA per
// SM; a persistent grid of one CTA per SM).
template <int N, int MODE>
void col_tma_z_n(const GridArgs& g, cudaStream_t s) {
  using Cfg = ColTmaZCfg<T, N>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_col_tma_z<T, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    attr = true;
  }
  ColTmaArgs<T> a;
  a.spec = reinterpret_cast<C*>(g.spec);
  a.g = reinterpret_cast<C*>(g.g);
  a.field_elems = g.field_elems;
  a.tw = reinterpret_cast<const C*>(g.tw_n);
  a.plane0 = reinterpret_cast<const C*>(g.plane0);
  a.dtab = reinterpret_cast<const T*>(g.dtab);
  a.wtab = reinterpret_cast<const T*>(g.wtab);
  a.gtab = reinterpret_cast<const T*>(g.gtab);
  a.fac = g.fac;
  a.fac_inv_du = g.fac_inv_du;
  a.coeff = g.green_coeff;
  a.status = g.status;
  const int items = Cfg::TILES_PER_ROW * N;
  const int grid = items < g.sm_count ? items : g.sm_count;
  if constexpr (sizeof(T) == 4 && MODE == kColFwdZ) {
    // FP32 forward: the form with its own exchange buffer (the next tile's copy
    // issued before the transform): 1.81 against 2.02 ms at 1024^3 on GB300.
    // The Green pass keeps k_col_tma_z, whose Green factors are computed while
    // its copy travels (2.27 against 2.46 ms with the factors computed inline
    // in a split-buffer form).  With bins_in_z it also sums the bins' power.
    if (g.bins_in_z) {
      using FC = ColTmaZFwdCfg<N, true>;
      static bool battr = false;
      if (!battr) {
        cudaFuncSetAttribute(k_col_tma_z_fwd<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FC::SMEM);
        battr = true;
      }
      a.thr = g.bin_thr;
      a.inv_lr = g.bin_inv_lr;
      a.nk = g.bin_nk;
      a.partials = g.bin_partials;
      k_col_tma_z_fwd<N, true><<<grid, FC::THREADS, FC::SMEM, s>>>(*g.tmap_z16, a);
    } else {
      using FC = ColTmaZFwdCfg<N, false>;
      static bool fattr = false;
      if (!fattr) {
        cudaFuncSetAttribute(k_col_tma_z_fwd<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FC::SMEM);
        fattr = true;
      }
      k_col_tma_z_fwd<N, false><<<grid, FC::THREADS, FC::SMEM, s>>>(*g.tmap_z16, a);
    }
    return;
  }
  k_col_tma_z<T, N, MODE><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*g.tmap_z16, a);
}

// One FFT pass of size N (pass: kPassXFwd .. kPassXInv, see nupm_internal.h).
template <int N>
void fft_pass_n(const GridArgs& g, int pass, cudaStream_t s) {
  if constexpr ((N & (N - 1)) == 0 && N >= 256) {   // TMA-staged z passes (tuning choice)
    if (g.wide_z == 2 && g.tmap_z16) {
      if (pass == kPassZFwd) { col_tma_z_n<N, kColFwdZ>(g, s); return; }
      if (pass == kPassZInv && g.fd_grad) { col_tma_z_n<N, kColInvZPhi>(g, s); return; }
      if (pass == kPassZInv) { col_tma_z_n<N, kColInvZGreen>(g, s); return; }
    }
  }
  if constexpr ((N & (N - 1)) == 0) {   // TMA column passes: power-of-two grids
  if (g.tmap_spec_y) {
    switch (pass) {
      case kPassYFwd: col_tma_n<N, kColFwdY>(g, g.tmap_spec_y, s); return;
      case kPassZFwd: col_tma_n<N, kColFwdZ>(g, g.tmap_spec_z, s); return;
      case kPassZInv: col_tma_n<N, kColInvZGreen>(g, g.tmap_spec_z, s); return;
      case kPassYInv: col_tma_n<N, kColInvYGrad>(g, g.tmap_g_y, s); return;
      default: break;
    }
  }
  }
  constexpr int M = N / 2;
  using RC = RowCfg<T, N>;
  const size_t row_smem = (size_t)RC::ROWS * RC::ROW_WORDS * sizeof(C);
  ensure_attrs<N>();
  const int64_t rows = (int64_t)N * N;
  const C* twn = reinterpret_cast<const C*>(g.tw_n);
  const C* twm = reinterpret_cast<const C*>(g.tw_m);
  (void)M;
  switch (pass) {
    case kPassXFwd:
      k_fft_x_fwd<T, N><<<(unsigned)(rows / RC::ROWS), RC::THREADS, row_smem, s>>>(
          reinterpret_cast<const unsigned long long*>(g.g), reinterpret_cast<C*>(g.spec), g.scale, twm, twn);
      break;
    case kPassXInv:
      // x with the x gradient on field 0 (phi -> d/dx phi); fields 1, 2 as they
      // are.  Real-space gradient: the potential alone.
      k_fft_x_inv<T, N><<<dim3((unsigned)(rows / RC::ROWS), 1, g.fd_grad ? 1 : 3), RC::THREADS, row_smem, s>>>(
          reinterpret_cast<C*>(g.g), g.field_elems, twm, twn, reinterpret_cast<const T*>(g.dtab),
          g.fd_grad ? 0 : 1);
      break;
    default: {
      // y passes narrow, z passes wide from N >= 256 on, unless tuned
      const bool zpass = pass == kPassZFwd || pass == kPassZInv;
      const int tuned = zpass ? g.wide_z : g.wide_y;
      const bool wide = tuned >= 0 ? tuned >= 1 : (zpass && N >= 256);
      if (wide) col_pass<N, ColWide<T, N>>(g, pass, s);
      else col_pass<N, ColNarrow<T, N>>(g, pass, s);
    }
  }
}

// Fused deposit + forward x pass of size N (rows sorted beforehand).
template <int N>
void deposit_fft_x_n(const GridArgs& g, const void* pos, bool keep, cudaStream_t s) {
  using F = FusedCfg<T, N>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_deposit_fft_x<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
    attr = true;
  }
  k_deposit_fft_x<T, N><<<dim3(N / F::TY, N / F::TZ), F::THREADS, F::SMEM, s>>>(
      g.rec, g.row_start, reinterpret_cast<C*>(g.spec), g.scale, reinterpret_cast<const C*>(g.tw_m),
      reinterpret_cast<const C*>(g.tw_n), keep ? reinterpret_cast<unsigned long long*>(g.g) : nullptr, g.status);
}

// Fused inverse x + interpolation + kick of size N (persistent grid).
template <int N>
void xinv_interp_n(const GridArgs& g, const void* pos, void* vel, double kick, void* acc_out, cudaStream_t s) {
  using X = XiCfg<T, N>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_xinv_interp<T, N, Quant<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::SMEM);
    attr = true;
  }
  const int items = (N / X::TZ) * (N / X::LY);
  const int grid = items < g.sm_count ? items : g.sm_count;
  k_xinv_interp<T, N, Quant<T>><<<grid, X::THREADS, X::SMEM, s>>>(
      reinterpret_cast<const C*>(g.g), g.field_elems, reinterpret_cast<const C*>(g.tw_m),
      reinterpret_cast<const C*>(g.tw_n), reinterpret_cast<const T*>(g.dtab), pos, g.np, g.delta, g.row_start,
      g.perm, reinterpret_cast<T*>(vel), (T)kick, reinterpret_cast<T*>(acc_out), g.status);
}

#define NUPM_DISPATCH(fn)                                  \
  switch (g.n) {                                           \
    case 16: fn<16>(g, pass, s); break;                    \
    case 32: fn<32>(g, pass, s); break;                    \
    case 64: fn<64>(g, pass, s); break;                    \
    case 128: fn<128>(g, pass, s); break;                  \
    case 256: fn<256>(g, pass, s); break;                  \
    case 512: fn<512>(g, pass, s); break;                  \
    case 1024: fn<1024>(g, pass, s); break;                \
    case 192: fn<192>(g, pass, s); break;                  \
    default: return PM_ERR_UNSUPPORTED;                    \
  }

int grid_blocks(int64_t work, int threads, int ctas_per_sm = 16) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)kSMs * ctas_per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

#define NUPM_CAT2(a, b) a##b
#define NUPM_CAT(a, b) NUPM_CAT2(a, b)
#define NUPM_FN(name) NUPM_CAT(name, NUPM_SFX)

int NUPM_FN(deposit)(const GridArgs& g, const void* pos, cudaStream_t s) {
  cudaMemsetAsync(g.g, 0, (size_t)g.n * g.n * g.n * sizeof(unsigned long long), s);
  if (g.np > 0)
    k_deposit<T><<<grid_blocks(g.np, 256), 256, 0, s>>>(pos, g.np, g.n, g.delta,
                                                       reinterpret_cast<unsigned long long*>(g.g), g.status);
  return PM_OK;
}

int NUPM_FN(row_sort)(const GridArgs& g, const void* pos, cudaStream_t s) {
  const int rows = g.n * g.n;
  cudaMemsetAsync(g.row_count, 0, (size_t)(rows + 1) * sizeof(int), s);
  const int blocks = grid_blocks(g.np, 256, g.part_ctas_per_sm);
  if (g.np > 0) k_row_count<T><<<blocks, 256, 0, s>>>(pos, g.np, g.n, g.delta, g.row_count, g.status);
  const int len = rows + 1;
  const int nb = (len + 2 * kScanBlock - 1) / (2 * kScanBlock);
  k_scan_blocks<<<nb, kScanBlock, 0, s>>>(g.row_count, g.row_start, g.scan_tot, len);
  k_scan_totals<<<1, kScanBlock, 0, s>>>(g.scan_tot, nb);
  k_scan_add<<<(len + 255) / 256, 256, 0, s>>>(g.row_start, g.scan_tot, len, g.row_cursor);
  if (g.np > 0)
    k_row_scatter<T><<<blocks, 256, 0, s>>>(pos, g.np, g.n, g.delta, g.row_cursor, g.perm, g.rec, g.inv);
  return PM_OK;
}

int NUPM_FN(deposit_fft_x)(const GridArgs& g, const void* pos, bool keep, cudaStream_t s) {
  switch (g.n) {
    case 16: deposit_fft_x_n<16>(g, pos, keep, s); break;
    case 32: deposit_fft_x_n<32>(g, pos, keep, s); break;
    case 64: deposit_fft_x_n<64>(g, pos, keep, s); break;
    case 128: deposit_fft_x_n<128>(g, pos, keep, s); break;
    case 256: deposit_fft_x_n<256>(g, pos, keep, s); break;
    case 512: deposit_fft_x_n<512>(g, pos, keep, s); break;
    case 1024: deposit_fft_x_n<1024>(g, pos, keep, s); break;
    case 192: deposit_fft_x_n<192>(g, pos, keep, s); break;
    default: return PM_ERR_UNSUPPORTED;
  }
  return PM_OK;
}

int NUPM_FN(fft_pass)(const GridArgs& g, int pass, cudaStream_t s) {
  NUPM_DISPATCH(fft_pass_n)
  return PM_OK;
}

int NUPM_FN(bins)(const GridArgs& g, bool lattice, int nk, const int* thr, float inv_lr, double kf,
                  double* partials, int nblk, double* out, cudaStream_t s) {
  const int nv = lattice ? 2 : 1;
  const int E = g.n / 64;
  const C* spec = reinterpret_cast<const C*>(g.spec);
  // one wave of resident CTAs (fewer than the partial rows when registers or
  // shared memory limit the residency), so no SM idles through a second wave
  auto wave = [&](const void* kern, size_t sh) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kBinWarps * 32, sh);
    const int resident = (o < 1 ? 1 : o) * g.sm_count;
    return resident < nblk ? resident : nblk;
  };
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    // FP32 power sums made by the forward z pass (one partial row per CTA of
    // its persistent grid): the packed x2 = 0 column here, then the reduce
    if (!lattice && g.bins_in_z) {
      const int zgrid = z_fwd_grid(g);
      const int nplane = (g.n + kPlaneBinWarps - 1) / kPlaneBinWarps;
      if (!bins_plane0<T>(g, nk, thr, inv_lr, partials, zgrid, nplane, s)) return PM_ERR_UNSUPPORTED;
      nblk = zgrid + nplane;
      done = true;
    }
    // FP32 power sums of grids with a bins tensor map: rows staged by TMA
    if (!done && !lattice && g.tmap_bins && (E == 2 || E == 4 || E == 8 || E == 16)) {
      decltype(&k_bin_power_tma<16>) kern = E == 2 ? k_bin_power_tma<2> : E == 4 ? k_bin_power_tma<4>
                                            : E == 8 ? k_bin_power_tma<8> : k_bin_power_tma<16>;
      const size_t sh = bin_tma_smem(nk, E);
      nblk = wave((const void*)kern, sh);
      kern<<<nblk, kBinWarps * 32, sh, s>>>(*g.tmap_bins, reinterpret_cast<const cx<float>*>(spec), g.n, nk, thr,
                                            inv_lr, partials, g.status);
      done = true;
    }
  }
  if (!done) {
    const size_t sh = kBinWarps * (size_t)nv * nk * sizeof(double) + (size_t)(nk + 1) * sizeof(int);
    if (lattice) {
      nblk = wave((const void*)k_bin_power<T, true>, sh);
      k_bin_power<T, true><<<nblk, kBinWarps * 32, sh, s>>>(spec, g.n, nk, thr, inv_lr, kf, partials);
    } else {
      nblk = wave((const void*)k_bin_power<T, false>, sh);
      k_bin_power<T, false><<<nblk, kBinWarps * 32, sh, s>>>(spec, g.n, nk, thr, inv_lr, kf, partials);
    }
  }
  k_bin_reduce<<<(nv * nk + 31) / 32, 1024, 0, s>>>(partials, nblk, nv * nk, out);
  return PM_OK;
}

int NUPM_FN(green)(const GridArgs& g, cudaStream_t s) {
  const int total = g.n * g.n;
  k_green_plane0<T><<<grid_blocks(total, 256), 256, 0, s>>>(
      reinterpret_cast<const C*>(g.spec), reinterpret_cast<C*>(g.plane0), g.n, reinterpret_cast<const T*>(g.gtab),
      reinterpret_cast<const T*>(g.wtab), g.fac, g.fac_inv_du, g.green_coeff);
  return PM_OK;
}

int NUPM_FN(interp)(const GridArgs& g, const void* pos, void* vel, double kick, void* acc_out, cudaStream_t s) {
  if (g.np > 0 && g.fd_grad && g.rows_ready && g.gather_rows == 2) {
    // forces in the sort's row order by sorted slot, then the velocities in particle order
    k_interp_rows_acc<T><<<(unsigned)((g.np + kGatherTPB * kGatherChunk - 1) / (kGatherTPB * kGatherChunk)),
                           kGatherTPB, 0, s>>>(g.rec, g.row_start, g.n, g.delta, reinterpret_cast<const T*>(g.g),
                                               reinterpret_cast<T*>(g.accs));
    k_kick_inv<T><<<grid_blocks(g.np, 256, g.part_ctas_per_sm), 256, 0, s>>>(
        g.inv, reinterpret_cast<const T*>(g.accs), g.np, reinterpret_cast<T*>(vel), (T)kick,
        reinterpret_cast<T*>(acc_out));
    return PM_OK;
  }
  if (g.np > 0 && g.fd_grad && g.rows_ready) {   // row order of the deposit's sort: a warp per row
    k_interp_rows_fd<T><<<(unsigned)(((int64_t)g.n * g.n + kRowsPerCta - 1) / kRowsPerCta), kGatherTPB, 0, s>>>(
        g.rec, g.row_start, g.perm, g.np, g.n, g.delta, reinterpret_cast<const T*>(g.g), reinterpret_cast<T*>(vel),
        (T)kick, reinterpret_cast<T*>(acc_out));
    return PM_OK;
  }
  if (g.np > 0 && g.fd_grad) {
    k_interp_kick_fd<T><<<(unsigned)((g.np + kGatherTPB * kGatherChunk - 1) / (kGatherTPB * kGatherChunk)),
                          kGatherTPB, 0, s>>>(
        pos, g.np, g.n, g.delta, reinterpret_cast<const T*>(g.g), reinterpret_cast<T*>(vel), (T)kick,
        reinterpret_cast<T*>(acc_out), g.status);
    return PM_OK;
  }
  if (g.np > 0)
    // 128-thread CTAs: the gather's ~96 registers per thread then fit 5 CTAs
    // (20 warps) per SM instead of 2 x 256 threads
    k_interp_kick<T><<<grid_blocks(g.np, 128, 2 * g.part_ctas_per_sm), 128, 0, s>>>(pos, g.np, g.n, g.delta,
                                                           reinterpret_cast<const T*>(g.g),
                                                           2 * g.field_elems, reinterpret_cast<T*>(vel), (T)kick,
                                                           reinterpret_cast<T*>(acc_out), g.status);
  return PM_OK;
}

int NUPM_FN(fd_field)(const GridArgs& g, int comp, void* dst, cudaStream_t s) {
  const int64_t total = (int64_t)g.n * g.n * g.n;
  k_fd_force_field<T><<<grid_blocks(total, 256), 256, 0, s>>>(reinterpret_cast<const T*>(g.g), g.n, comp, g.delta,
                                                             reinterpret_cast<T*>(dst));
  return PM_OK;
}

int NUPM_FN(xinv_interp)(const GridArgs& g, const void* pos, void* vel, double kick, void* acc_out,
                         cudaStream_t s) {
  switch (g.n) {
    case 16: xinv_interp_n<16>(g, pos, vel, kick, acc_out, s); break;
    case 32: xinv_interp_n<32>(g, pos, vel, kick, acc_out, s); break;
    case 64: xinv_interp_n<64>(g, pos, vel, kick, acc_out, s); break;
    case 128: xinv_interp_n<128>(g, pos, vel, kick, acc_out, s); break;
    case 256: xinv_interp_n<256>(g, pos, vel, kick, acc_out, s); break;
    case 512: xinv_interp_n<512>(g, pos, vel, kick, acc_out, s); break;
    case 1024: xinv_interp_n<1024>(g, pos, vel, kick, acc_out, s); break;
    default: return PM_ERR_UNSUPPORTED;
  }
  return PM_OK;
}

int NUPM_FN(drift)(const GridArgs& g, void* pos, const void* vel, double ds, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (g.np > 0 && (g.np & 3) == 0 && ((uintptr_t)pos & 15) == 0 && ((uintptr_t)vel & 15) == 0) {
      k_drift4<<<grid_blocks(g.np / 4, 256, 8), 256, 0, s>>>(reinterpret_cast<int32_t*>(pos),
                                                             reinterpret_cast<const float*>(vel), g.np, g.n,
                                                             (float)(ds / g.delta), g.status);
      return PM_OK;
    }
  }
  if (g.np > 0)
    k_drift<T><<<grid_blocks(g.np, 256, 8), 256, 0, s>>>(pos, reinterpret_cast<const T*>(vel), g.np, g.n, g.box, ds,
                                                          (float)(ds / g.delta), g.status);
  return PM_OK;
}

int NUPM_FN(unpack)(const GridArgs& g, void* dst, cudaStream_t s) {
  const int64_t total = (int64_t)g.n * g.n * (g.n / 2 + 1);
  k_unpack_spec<T><<<grid_blocks(total, 256), 256, 0, s>>>(reinterpret_cast<const C*>(g.spec),
                                                          reinterpret_cast<C*>(dst), g.n);
  return PM_OK;
}

#undef NUPM_FN
#undef NUPM_CAT
#undef NUPM_CAT2
#undef NUPM_DISPATCH

}  // namespace nupm
