"""CPU FP64 oracle for the particle-mesh kick with linear-response neutrinos.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
restatement of what the GPU path computes.  Only the test-suite, the smoke
check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import or run it.  The product path (the CUDA library and its Python binding)
never imports it and never falls back to it; the two share no code.

Paper: Ali-Haimoud & Bird, "An efficient implementation of massive neutrinos
in non-linear structure formation simulations" (arXiv:1209.0461).  Every
function names the section / equation it restates.

Units (H0 = 1): lengths in Mpc/h, time in 1/H0, velocities u = a^2 dx/dt in
units of H0 * Mpc/h (= 100 km/s), conformal time tau and superconformal time
s = int dtau / a in 1/H0 (Sec. 3.2).  With c = 1 inside the free-streaming
argument, x = k * (c/H0) * (s - s') * T_nu0 / m_nu (App. C: x = X T_nu0,
X = k (s - s') / m from Eq. I.def / Eq. delta.final).

Parity status: every function below is pinned by a test in
``tests/test_oracle_*.py`` against closed forms, printed values, brute force or
an independent route (see each function's docstring, "Pinned by").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import integrate, special

# --------------------------------------------------------------------------
# Constants (Sec. 2.1)
# --------------------------------------------------------------------------
T_NU0_EV = 1.68e-4          # Sec. 2.1: T_nu,0 = 1.95 K = 1.68e-4 eV (value as printed)
OMEGA_NU_EV = 93.14         # Sec. 2.1: Omega_nu h^2 = sum m_nu / 93.14 eV
C_OVER_H0 = 2997.92458      # c / H0 in Mpc/h
WEIGHT_BITS = 16            # fixed-point CIC weight resolution per axis
WEIGHT_ONE = 1 << WEIGHT_BITS
MASS_ONE = WEIGHT_ONE ** 3  # 2^48: one particle's total deposit
ZETA3 = float(special.zeta(3.0))


def omega_nu_from_mass(m_nu_total_ev: float, h: float) -> float:
    """Omega_nu = M_nu / (93.14 eV h^2) (Sec. 2.1, f_nu definition).

    Pinned by: tests check the paper's printed f_nu ~ 0.022 for M_nu = 0.3 eV,
    Omega_M h^2 = 0.147.
    """
    return m_nu_total_ev / (OMEGA_NU_EV * h * h)


# --------------------------------------------------------------------------
# Free-streaming kernel I(x)  (Eq. I.def; App. C series and Eq. fit)
# --------------------------------------------------------------------------
def nu_I(x) -> np.ndarray:
    """Fermi-Dirac free-streaming kernel I(x), exact, from the App. C series

        I(x) = 4 / (3 zeta(3)) * sum_{n>=1} (-1)^{n+1} n / (n^2 + x^2)^2,

    which is the closed evaluation of Eq. I.def with f0 the relativistic
    Fermi-Dirac distribution (Sec. 4.1, g = 2) and x = X T_nu0.

    The alternating series is summed directly up to N terms (N well past the
    peak of the terms at n ~ x / sqrt 3) and the remaining tail is taken by
    repeated averaging of the last partial sums (Euler's transform of an
    alternating series).  x values are grouped by magnitude so each group
    uses only as many terms as it needs.

    Pinned by: I(0) = 1; small-x slope 5 zeta(5) / (2 zeta(3)) and large-x
    limit 1 / (3 zeta(3) x^4) (App. C); brute-force partial sums with 10^6
    terms; quadrature of Eq. I.def; int_0^inf x I(x) dx = 2 ln 2 / (3 zeta 3)
    (Sec. 3.3.2 with Eq. v2).
    """
    x = np.abs(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    flat_x = x.ravel()
    flat_o = out.ravel()
    # group by needed term count: N = 48 + 4 x, rounded up to a power of two
    need = 48.0 + 4.0 * flat_x
    grp = np.ceil(np.log2(need)).astype(np.int64)
    n_avg = 20
    for g in np.unique(grp):
        sel = np.nonzero(grp == g)[0]
        nterm = int(2 ** g) + n_avg
        n = np.arange(1, nterm + 1, dtype=np.float64)
        xs = flat_x[sel][:, None]
        sign = np.where(n % 2 == 1, 1.0, -1.0)
        terms = sign * n / (n * n + xs * xs) ** 2
        nbase = nterm - n_avg
        base = terms[:, :nbase].sum(axis=1)
        # partial sums S_nbase .. S_nterm, then n_avg rounds of averaging
        ps = base[:, None] + np.concatenate(
            [np.zeros((len(sel), 1)), np.cumsum(terms[:, nbase:], axis=1)], axis=1)
        for _ in range(n_avg):
            ps = 0.5 * (ps[:, 1:] + ps[:, :-1])
        flat_o[sel] = ps[:, 0]
    return out * (4.0 / (3.0 * ZETA3))


def nu_I_fit(x) -> np.ndarray:
    """Fitting formula for I(x) (App. C, Eq. fit).

    Pinned by: the paper's stated accuracy against the exact series
    (absolute <~ 0.07%, relative <~ 1% on 0 <= x <= 2).
    """
    x = np.abs(np.asarray(x, dtype=np.float64))
    x2 = x * x
    num = 1.0 + 0.0168 * x2 + 0.0407 * x2 * x2
    den = 1.0 + 2.1734 * x2 + 1.6787 * np.power(x, 4.1811) + 0.1467 * x2 ** 4
    return num / den


# --------------------------------------------------------------------------
# Background (Sec. 3.2 superconformal time; Sec. 3.1 kick/drift)
# --------------------------------------------------------------------------
def hubble(a, omega_m):
    """H(a)/H0.  ``omega_m`` a number: flat matter + Lambda,
    sqrt(Om a^-3 + 1 - Om).  A ``Cosmo``: the same from its Omega_M, or, with
    ``relativistic`` set, the background of Sec. 4.4 (``Cosmo.e2``)."""
    a = np.asarray(a, dtype=np.float64)
    if isinstance(omega_m, Cosmo):
        if omega_m.relativistic:
            return np.sqrt(omega_m.e2(a))
        omega_m = omega_m.omega_m
    return np.sqrt(omega_m / a ** 3 + (1.0 - omega_m))


# Radiation today (Sec. 4.4 adds it to the background): photons at
# T_cmb = 2.7255 K, Omega_gamma h^2 = 2.4728e-5; each massless neutrino species
# carries (7/8)(4/11)^{4/3} of the photon density (T_nu / T_gamma = (4/11)^{1/3}).
OMEGA_GAMMA_H2 = 2.4728e-5
NU_TO_GAMMA = 7.0 / 8.0 * (4.0 / 11.0) ** (4.0 / 3.0)
N_NU_SPECIES = 3
_FD_X, _FD_W = np.polynomial.legendre.leggauss(32)


def nu_energy_ratio(y):
    """rho_nu(a) / rho_nu,NR(a) of one massive species, from Eq. relativistic:
    rho = a^-3 int eps(q, a) f0(q) 4 pi q^2 dq with eps = sqrt(m^2 + q^2/a^2)
    and f0 the relativistic Fermi-Dirac distribution at T_nu0, against its
    non-relativistic limit a^-3 m int f0 4 pi q^2 dq.  With x = q / T_nu0 and
    y = m a / T_nu0,

        R(y) = int_0^inf sqrt(1 + x^2/y^2) x^2 / (e^x + 1) dx / ((3/2) zeta(3)),

    (3/2) zeta(3) being int x^2 / (e^x + 1) dx.  Composite 32-point
    Gauss-Legendre on [0, 64] split at 1, 2, 4, ..., 64 and at 2y, 4y, 8y, ...
    (the square root's poles x = +-iy then lie at least a panel half-width
    from every panel); the tail beyond x = 64 is below 1e-24 of the total.

    Pinned by: R -> 1 + (15 zeta(5) / zeta(3)) / (2 y^2) at large y; y R ->
    7 pi^4 / (180 zeta(3)) at small y (the relativistic fermion energy density
    (7/8)(pi^2/15) T^4 per species); adaptive quadrature at y = 0.3 .. 30.
    """
    y = np.asarray(y, dtype=np.float64)
    yf = y.reshape(-1, 1)
    fixed = np.broadcast_to(2.0 ** np.arange(-1, 7, dtype=np.float64), (yf.shape[0], 8)).copy()
    fixed[:, 0] = 0.0
    geo = np.minimum(2.0 * yf * 2.0 ** np.arange(24, dtype=np.float64), 64.0)
    edges = np.sort(np.concatenate([fixed, geo], axis=1), axis=1)        # [ny, 32]
    lo, hi = edges[:, :-1, None], edges[:, 1:, None]
    half = 0.5 * (hi - lo)
    x = lo + half * (_FD_X + 1.0)
    yy = yf[:, :, None]
    f = np.sqrt(1.0 + (x / yy) ** 2) * x * x / (np.exp(x) + 1.0)
    val = (half * f * _FD_W).sum(axis=(1, 2))
    return (val / (1.5 * ZETA3)).reshape(y.shape)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(64)


def delta_s(a_lo, a_hi, omega_m):
    """s(a_hi) - s(a_lo) = int_{a_lo}^{a_hi} da / (a^3 H)  (Sec. 3.2: ds = dtau/a,
    dtau = da / (a^2 H)).

    64-point Gauss-Legendre in ln a (integrand a^-2 / H, smooth); vectorised
    over array arguments.  Computed directly as a difference-free integral so
    that s - s' stays accurate when a' -> a.

    Pinned by: scipy adaptive quad; Einstein-de Sitter closed form
    2 (a_lo^-1/2 - a_hi^-1/2).
    """
    a_lo = np.asarray(a_lo, dtype=np.float64)
    a_hi = np.asarray(a_hi, dtype=np.float64)
    u0 = np.log(a_lo)[..., None]
    # ln(a_hi / a_lo) via log1p of the exact difference: no cancellation when
    # a_hi -> a_lo
    half = 0.5 * np.log1p((a_hi - a_lo) / a_lo)[..., None]
    u = u0 + half * (_GL_X + 1.0)
    a = np.exp(u)
    f = 1.0 / (a * a * hubble(a, omega_m))     # da/(a^3 H) = d ln a / (a^2 H)
    return (half * (f * _GL_W)).sum(axis=-1)


def s_of_a(a, a_init: float, omega_m: float):
    """Superconformal time s(a) = int_{a_init}^{a} da / (a^3 H) (Sec. 3.2)."""
    return delta_s(np.full_like(np.asarray(a, dtype=np.float64), a_init), a, omega_m)


def kick_factor(a0: float, a1: float, omega_m) -> float:
    """K = int_{a0}^{a1} dt = int da / (a H): the velocity u = a^2 dx/dt obeys
    du/dt = -grad phi (Eq. dot.q.2 with q = m u).  Adaptive quadrature.

    Pinned by: EdS closed form (2/3)(a1^{3/2} - a0^{3/2}).
    """
    val, _ = integrate.quad(lambda a: 1.0 / (a * float(hubble(a, omega_m))), a0, a1,
                            epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def drift_factor(a0: float, a1: float, omega_m) -> float:
    """Delta s = int da / (a^3 H): dx/dt = u / a^2 (Sec. 3.1 definition of q)."""
    val, _ = integrate.quad(lambda a: 1.0 / (a ** 3 * float(hubble(a, omega_m))), a0, a1,
                            epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def free_streaming_k(a: float, m_ev: float, omega_m: float) -> float:
    """Free-streaming wavenumber k_fs(a) = (3/2 Omega_M(a) <v^-2>)^{1/2} a H in
    h/Mpc (Eq. kfs-formal), with <v^-2> = 2 ln 2 / (3 zeta 3) (m a / T_nu0)^2
    (Eq. v2, c = 1) and Omega_M(a) = Omega_M a^-3 / H^2.  Used only by tests
    (small-scale limit of Sec. 3.3.2, App. A).

    Pinned by: the numerical forms of Eq. kfs (0.08 h/Mpc) and Eq. v2
    (810 km/s).
    """
    H = float(hubble(a, omega_m))
    om_a = omega_m / a ** 3 / H ** 2
    v2 = 2.0 * math.log(2.0) / (3.0 * ZETA3) * (m_ev * a / T_NU0_EV) ** 2
    return math.sqrt(1.5 * om_a * v2) * a * H / C_OVER_H0


# --------------------------------------------------------------------------
# Particle quantisation and CIC deposit (Sec. 4.3 step (ii): the Fourier-
# transformed CDM density needed for the long-range PM force)
# --------------------------------------------------------------------------
def quantise_positions_f64(pos: np.ndarray, box: float, ngrid: int):
    """FP64 comoving positions [3, Np] -> (cell [3,Np] int64 in [0,N), w [3,Np]).

    u = x / (L/N); c = floor(u); w = floor((u - c) * 2^16); c wrapped mod N.
    """
    delta = box / ngrid
    u = np.asarray(pos, dtype=np.float64) / delta
    c = np.floor(u)
    o = u - c
    w = np.floor(o * WEIGHT_ONE).astype(np.int64)
    c = np.mod(c.astype(np.int64), ngrid)
    return c, w


def quantise_positions_cell(cell: np.ndarray, off: np.ndarray, ngrid: int):
    """Cell-index + FP32-offset positions -> (cell mod N, w = floor(off * 2^16)).

    Offsets must lie in [0, 1); raises ValueError otherwise.
    """
    off = np.asarray(off, dtype=np.float32)
    if np.any(~np.isfinite(off)) or np.any(off < 0) or np.any(off >= 1):
        raise ValueError("offsets must lie in [0, 1)")
    w = np.floor(off.astype(np.float64) * WEIGHT_ONE).astype(np.int64)
    c = np.mod(np.asarray(cell, dtype=np.int64), ngrid)
    return c, w


def _corner_weights(w):
    """Per-axis fixed-point weights: (2^16 - w) at cell c, w at cell c + 1."""
    return (WEIGHT_ONE - w, w)


def cic_deposit(c: np.ndarray, w: np.ndarray, ngrid: int) -> np.ndarray:
    """Fixed-point cloud-in-cell deposit: F[z, y, x] (int64), each particle
    adding wx*wy*wz (product of per-axis 16-bit weights, total 2^48) to the 8
    corner nodes.  Integer sums are exact, so the result is order-independent.

    Pinned by: exact mass conservation sum F = Np 2^48; a hand-computed single
    particle; brute-force per-particle loop.
    """
    n = ngrid
    grid = np.zeros(n * n * n, dtype=np.int64)
    wx, wy, wz = (_corner_weights(w[0]), _corner_weights(w[1]), _corner_weights(w[2]))
    for dz in (0, 1):
        iz = (c[2] + dz) % n
        for dy in (0, 1):
            iy = (c[1] + dy) % n
            for dx in (0, 1):
                ix = (c[0] + dx) % n
                wt = wx[dx] * wy[dy] * wz[dz]
                np.add.at(grid, (iz * n + iy) * n + ix, wt)
    return grid.reshape(n, n, n)


def cic_deposit_cells(c: np.ndarray, w: np.ndarray, ngrid: int, cells: np.ndarray) -> np.ndarray:
    """The deposit F of ``cic_deposit`` at the flat nodes ``cells`` ((z N + y)
    N + x) only, without the N^3 grid: F(t) is the sum over particles p and
    corners d in {0,1}^3 with (c_p + d) mod N = t of wx[dx] wy[dy] wz[dz].
    Only particles whose base cell is t - d for some d can contribute, so those
    are picked first (int64 sums, exact).

    Pinned by: equal to cic_deposit at every sampled node (wrapped nodes too).
    """
    n = ngrid
    cells = np.asarray(cells, dtype=np.int64).reshape(-1)
    tz, ty, tx = cells // (n * n), (cells // n) % n, cells % n
    base = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                base.append((((tz - dz) % n) * n + (ty - dy) % n) * n + (tx - dx) % n)
    flat = (c[2].astype(np.int64) * n + c[1]) * n + c[0]
    sel = np.nonzero(np.isin(flat, np.unique(np.concatenate(base)), kind="table"))[0]
    cs, ws = c[:, sel], w[:, sel]
    wx, wy, wz = (_corner_weights(ws[0]), _corner_weights(ws[1]), _corner_weights(ws[2]))
    out = np.zeros(cells.size, dtype=np.int64)
    for dz in (0, 1):
        iz = (cs[2] + dz) % n
        for dy in (0, 1):
            iy = (cs[1] + dy) % n
            for dx in (0, 1):
                ix = (cs[0] + dx) % n
                node = (iz * n + iy) * n + ix
                wt = wx[dx] * wy[dy] * wz[dz]
                for i, t in enumerate(cells):
                    out[i] += int(wt[node == t].sum())
    return out


def density_modes(c: np.ndarray, w: np.ndarray, ngrid: int, npart: int, kz, ky, kx,
                  chunk: int = 1 << 22) -> np.ndarray:
    """delta(k) of ``forward_fft(density_contrast(cic_deposit(c, w)))`` at the
    given integer modes (kz, ky signed, kx in [0, N/2]) without the grid: by
    linearity of the DFT,
      sum_x F(x) e^{-2 pi i k.x / N}
        = sum_p prod_axes [W0 e^{-2 pi i k_a c_a / N} + W1 e^{-2 pi i k_a (c_a+1) / N}]
    (the corner weight is the product of the per-axis weights W0 = 2^16 - w,
    W1 = w), then delta(k) = that sum N^3 / (Np 2^48) - N^3 [k = 0].  The
    phases come from a table of e^{-2 pi i m / N} at the exact integer index
    m = (k c) mod N.  The sum over particles runs in chunks as one matrix
    product per chunk (library step): rows z-factors, columns the (y, x)
    factor products.  Plain PyTorch CPU ops (threaded) do the chunk arithmetic.

    Pinned by: equal to a brute-force DFT of the deposited density, and to the
    FFT route, at sampled modes.
    """
    import torch
    n = ngrid
    kz, ky, kx = (np.asarray(v, dtype=np.int64).reshape(-1) for v in (kz, ky, kx))
    uz, iz_of = np.unique(kz, return_inverse=True)
    uy, iy_of = np.unique(ky, return_inverse=True)
    ux, ix_of = np.unique(kx, return_inverse=True)
    unit = torch.exp(-2j * math.pi * torch.arange(n, dtype=torch.float64) / n)
    fr = [torch.from_numpy(u) for u in (ux, uy, uz)]
    acc = torch.zeros((uz.size, uy.size * ux.size), dtype=torch.complex128)

    def axis_factor(ca, wa, freqs):
        ph = unit[torch.remainder(ca[:, None] * freqs[None, :], n)]
        step = unit[torch.remainder(freqs, n)]
        return ph * ((WEIGHT_ONE - wa).double()[:, None] + wa.double()[:, None] * step[None, :])

    total = c.shape[1]
    for s0 in range(0, total, chunk):
        s1 = min(s0 + chunk, total)
        cc = torch.from_numpy(np.ascontiguousarray(c[:, s0:s1], dtype=np.int64))
        ww = torch.from_numpy(np.ascontiguousarray(w[:, s0:s1], dtype=np.int64))
        fx = axis_factor(cc[0], ww[0], fr[0])
        fy = axis_factor(cc[1], ww[1], fr[1])
        fz = axis_factor(cc[2], ww[2], fr[2])
        yx = (fy[:, :, None] * fx[:, None, :]).reshape(fx.shape[0], -1)
        acc += fz.T @ yx
    val = acc.numpy()[iz_of, iy_of * ux.size + ix_of]
    out = val * (float(n) ** 3 / (float(npart) * MASS_ONE))
    out[(kz == 0) & (ky == 0) & (kx == 0)] -= float(n) ** 3
    return out


def density_contrast(F: np.ndarray, npart: int) -> np.ndarray:
    """delta = F N^3 / (Np 2^48) - 1 in FP64 (mean particle count per node is
    Np / N^3)."""
    n = F.shape[0]
    return F.astype(np.float64) * (float(n) ** 3 / (float(npart) * MASS_ONE)) - 1.0


def forward_fft(delta: np.ndarray) -> np.ndarray:
    """Unnormalised forward real 3-D DFT, half spectrum over x: spec[kz, ky, kx],
    kx in [0, N/2].  numpy.fft.rfftn serves as the library step.

    Pinned by: brute-force DFT at 8^3; Parseval.
    """
    return np.fft.rfftn(delta)


# --------------------------------------------------------------------------
# Power-spectrum bins (Sec. 4.2-4.3: P_cdm(k, tau) per |k| bin)
# --------------------------------------------------------------------------
def bin_thresholds(ngrid: int, n_kbins: int) -> np.ndarray:
    """Integer n^2 thresholds T_b = ceil((e_b L / 2 pi)^2), b = 0..n_kbins, for
    log-spaced edges e_b = k_min (k_max/k_min)^(b/nk), k_min = 2 pi / L,
    k_max = sqrt(3) pi N / L (1 + 1e-12).  A mode with integer n^2 lies in bin
    b iff T_b <= n^2 < T_{b+1}; a mode exactly on an edge goes to the upper
    bin.  n^2 = 0 (the mean) is in no bin."""
    r = math.sqrt(3.0) * ngrid / 2.0 * (1.0 + 1e-12)
    b = np.arange(n_kbins + 1, dtype=np.float64)
    return np.ceil(np.power(r, 2.0 * b / n_kbins)).astype(np.int64)


def mode_indices(ngrid: int):
    """Signed integer frequencies (iz, iy, ix) of the half spectrum, broadcastable."""
    n = ngrid
    f = np.fft.fftfreq(n, d=1.0 / n).astype(np.int64)   # 0..N/2-1, -N/2..-1
    ix = np.arange(n // 2 + 1, dtype=np.int64)
    return f[:, None, None], f[None, :, None], ix[None, None, :]


def bin_power(spec: np.ndarray, box: float, n_kbins: int):
    """Binned power spectrum of the half spectrum ``spec`` (Sec. 4.3 step (ii)).

    Weight w = 1 on the kx = 0 and kx = N/2 planes, 2 elsewhere (each counts
    a mode and its conjugate).  Returns dict with per-bin
      count = sum w, ksum = sum w |k|, psum = sum w |delta_k|^2,
      P = psum / count * L^3 / N^6   [(Mpc/h)^3],  k = ksum / count,
      nonempty mask.

    Pinned by: a single plane wave lands in one bin with known power; mode
    counts equal a brute-force lattice enumeration.
    """
    n = spec.shape[0]
    iz, iy, ix = mode_indices(n)
    return bin_power_modes(spec, iz, iy, ix, n, box, n_kbins)


def bin_power_modes(spec, iz, iy, ix, ngrid: int, box: float, n_kbins: int):
    """``bin_power`` over an explicit set of half-spectrum modes (iz, iy, ix
    broadcastable to spec): the same weights, thresholds and sums.  Over the
    whole half lattice it is bin_power; over all modes of some bins it gives
    those bins' entries exactly."""
    n = ngrid
    n2 = iz * iz + iy * iy + ix * ix
    w = np.where((ix == 0) | (ix == n // 2), 1.0, 2.0) * np.ones_like(n2, dtype=np.float64)
    T = bin_thresholds(n, n_kbins)
    b = np.searchsorted(T, n2, side="right") - 1
    valid = (n2 > 0) & (b >= 0) & (b < n_kbins)
    bb = b[valid]
    ww = w[valid]
    kf = 2.0 * math.pi / box
    kmag = kf * np.sqrt(n2[valid].astype(np.float64))
    p2 = (np.abs(spec[valid]) ** 2)
    count = np.bincount(bb, weights=ww, minlength=n_kbins)
    ksum = np.bincount(bb, weights=ww * kmag, minlength=n_kbins)
    psum = np.bincount(bb, weights=ww * p2, minlength=n_kbins)
    ne = count > 0
    P = np.zeros(n_kbins)
    k = np.zeros(n_kbins)
    P[ne] = psum[ne] / count[ne] * box ** 3 / float(n) ** 6
    k[ne] = ksum[ne] / count[ne]
    return dict(count=count, ksum=ksum, psum=psum, P=P, k=k, nonempty=ne, T=T)


# --------------------------------------------------------------------------
# Neutrino linear response (Eq. P-final, Eq. deltaI-nu, Sec. 4.3 (iii), App. B)
# --------------------------------------------------------------------------
@dataclass
class Cosmo:
    """Cosmology of the kick.  Omega_M = omega_cdm + omega_nu (baryons folded
    into cdm); flat, Omega_L = 1 - Omega_M.  m_nu_ev lists the species masses."""
    omega_cdm: float
    omega_nu: float
    h: float
    m_nu_ev: tuple = ()
    a_init: float = 0.02
    relativistic: bool = False   # Sec. 4.4 background: rho_nu(a) of Eq. relativistic + radiation

    @property
    def omega_m(self) -> float:
        return self.omega_cdm + self.omega_nu

    @property
    def f_nu(self) -> float:
        return self.omega_nu / self.omega_m

    @property
    def omega_r(self) -> float:
        """Radiation today: photons plus the massless neutrino species (of
        N_NU_SPECIES, those not listed with a mass)."""
        n_massive = sum(1 for m in self.m_nu_ev if m > 0) if self.omega_nu > 0 else 0
        return OMEGA_GAMMA_H2 / self.h ** 2 * (1.0 + (N_NU_SPECIES - n_massive) * NU_TO_GAMMA)

    def e2(self, a):
        """(H/H0)^2 of the Sec. 4.4 background: CDM (a^-3), each massive
        species Omega_nu,i R(m_i a / T_nu0) a^-3 (Eq. relativistic), radiation
        Omega_r a^-4, and Lambda closing the universe at a = 1."""
        a = np.asarray(a, dtype=np.float64)
        out = self.omega_cdm / a ** 3 + self.omega_r / a ** 4
        nu_today = 0.0
        masses = np.asarray(self.m_nu_ev, dtype=np.float64)
        if self.omega_nu > 0 and masses.size and masses.sum() > 0:
            for m, wi in zip(masses, self.species_weights()):
                if m > 0:
                    onu = self.omega_nu * wi
                    out = out + onu * nu_energy_ratio(m * a / T_NU0_EV) / a ** 3
                    nu_today += onu * float(nu_energy_ratio(m / T_NU0_EV))
        elif self.omega_nu > 0:
            out = out + self.omega_nu / a ** 3
            nu_today = self.omega_nu
        return out + (1.0 - self.omega_cdm - nu_today - self.omega_r)

    def species_weights(self):
        """Omega_nu,i / Omega_nu = m_i / M_nu (Sec. 2.1 per species).

        Pinned by: a light second species (m_2 = m_1/50) leaves the heavy
        species' response scaled by m_1/M_nu, in either order; a three-mass
        hierarchy equals the mass-weighted sum of single-species responses.
        """
        m = np.asarray(self.m_nu_ev, dtype=np.float64)
        tot = m.sum()
        return m / tot if tot > 0 else np.zeros_like(m)


def _interp_lna(lna_nodes, vals, lna):
    """Piecewise-linear in ln a between nodes; constant before the first node.
    vals: [n_nodes, nb]; lna: array -> [len(lna), nb]."""
    lna = np.atleast_1d(lna)
    out = np.empty((lna.size, vals.shape[1]))
    for i, u in enumerate(lna):
        if len(lna_nodes) == 1 or u <= lna_nodes[0]:
            out[i] = vals[0]
            continue
        j = np.searchsorted(lna_nodes, u, side="right") - 1
        j = min(max(j, 0), len(lna_nodes) - 2)
        t = (u - lna_nodes[j]) / (lna_nodes[j + 1] - lna_nodes[j])
        out[i] = vals[j] + (vals[j + 1] - vals[j]) * t
    return out


def response_integral(kb, a, cosmo: Cosmo, m_ev: float, a_nodes, h_nodes,
                      I_func=nu_I, epsrel=1e-11):
    """Integral term of Eq. P-final for one species:

        J(k) = (3/2) Omega_M H0^2 int_{tau_i}^{tau} I[k (s - s') / m] (s - s')
               P_M^{1/2}(k, tau') dtau',       dtau' = da' / (a'^2 H(a')),

    with P_M^{1/2}(k, a') linear in ln a' through the nodes (a_nodes, h_nodes)
    (h_nodes [n_nodes, nb]) and constant on [a_i, a_nodes[0]].  The last node
    must be the current epoch a.  Integrated in ln a' by vector-valued
    adaptive quadrature (scipy quad_vec, the nodes as break points) to
    ``epsrel``.

    Pinned by: EdS with I == 1 and constant P_M^{1/2} gives the closed form
    3 c [ln(a/a_i) - 2 (1 - sqrt(a_i/a))]; a brute-force fine composite rule
    in the superconformal-time variable; the small-scale limit (k_fs/k)^2.
    """
    kb = np.asarray(kb, dtype=np.float64)
    om = cosmo.omega_m
    bg = cosmo                                          # background of s(a) and H(a)
    kappa = kb * C_OVER_H0 * T_NU0_EV / m_ev            # x = kappa (s - s')
    lna_nodes = np.log(np.asarray(a_nodes, dtype=np.float64))
    h_nodes = np.asarray(h_nodes, dtype=np.float64)
    ai = cosmo.a_init

    def integrand(u):
        ap = math.exp(u)
        ds = float(delta_s(ap, a, bg))
        h = _interp_lna(lna_nodes, h_nodes, u)[0]
        x = kappa * ds
        return I_func(x) * ds * h / (ap * float(hubble(ap, bg)))   # dtau'/dln a' = 1/(a' H)

    u_lo, u_hi = math.log(ai), math.log(a)
    if u_hi <= u_lo:
        return np.zeros_like(kb)
    inner = [u for u in lna_nodes if u_lo < u < u_hi]
    val, _ = integrate.quad_vec(integrand, u_lo, u_hi, epsabs=0.0, epsrel=epsrel,
                                norm="max", limit=200000, points=inner or None)
    return 1.5 * om * val


def ic_term(kb, a, cosmo: Cosmo, m_ev: float, sqrtPnu_init, theta_over_delta_init,
            I_func=nu_I):
    """Initial-condition term of Eq. P-final (Eq. deltaI-nu):
    I_{s_i,s} P_nu,i^{1/2}(k) {1 - (s - s_i) a_i [theta/delta]_i(k)}."""
    kb = np.asarray(kb, dtype=np.float64)
    ds = float(delta_s(cosmo.a_init, a, cosmo))
    x = kb * C_OVER_H0 * T_NU0_EV / m_ev * ds
    return I_func(x) * np.asarray(sqrtPnu_init) * (
        1.0 - ds * cosmo.a_init * np.asarray(theta_over_delta_init))


def nu_K(y) -> np.ndarray:
    """The l = 1 term of Eq. deltaI-multipole for the paper's initial moments
    (delta f_1 = (df_0/dq) m a_i theta / k, Sec. 4.1), as a function of
    y = k (s - s_i) T_nu0 / m:

        K(y) = -(1/y) int_0^inf u^2 f'(u) j_1(u y) du / int_0^inf u^2 f(u) du,
        f(u) = 1 / (e^u + 1),

    so that the term is -P_nu,i^{1/2} a_i [theta/delta]_i (s - s_i) K(y).
    Evaluated directly as a momentum integral of j_1 (QUADPACK): for y < 1
    the integrand with j_1 itself, for y >= 1 the Fourier form
    j_1(z) = sin z / z^2 - cos z / z with sine and cosine weights.

    Pinned by: K(0) = 1 and the small-y series 1 - (5 zeta(5) / (2 zeta(3)))
    y^2; K = I of Eq. I.def (the integration by parts of Sec. 4.1 is exact
    for these moments: d/dz [z^2 j_1(z)] = z^2 j_0(z)), checked at y from
    1e-2 to 1e2 against the App. C series of I.
    """
    shape = np.shape(y)
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    out = np.empty_like(y)
    norm = 1.5 * ZETA3

    def fp(u):                                   # f'(u) = -e^{-u} / (1 + e^{-u})^2
        e = math.exp(-u)
        return -e / (1.0 + e) ** 2

    for i, yy in enumerate(y.ravel()):
        if yy == 0.0:
            out.flat[i] = 1.0
            continue
        if yy < 1.0:
            v, _ = integrate.quad(lambda u: u * u * fp(u) * special.spherical_jn(1, u * yy), 0.0, 80.0,
                                  epsabs=0.0, epsrel=1e-13, limit=400)
            out.flat[i] = -v / (yy * norm)
        else:
            s1, _ = integrate.quad(fp, 0.0, 80.0, weight="sin", wvar=yy, epsabs=1e-15, epsrel=1e-13, limit=400)
            c1, _ = integrate.quad(lambda u: u * fp(u), 0.0, 80.0, weight="cos", wvar=yy, epsabs=1e-15,
                                   epsrel=1e-13, limit=400)
            out.flat[i] = -(s1 / (yy * yy) - c1 / yy) / (yy * norm)
    return out.reshape(shape)


def ic_term_multipole(kb, a, cosmo: Cosmo, m_ev: float, sqrtPnu_init, theta_over_delta_init, I_func=nu_I):
    """The initial-condition term by Eq. deltaI-multipole with the l = 0, 1
    moments of Sec. 4.1 (before its integration by parts):
    P_nu,i^{1/2} {I(y) - (s - s_i) a_i [theta/delta]_i K(y)}, K from the j_1
    integral (nu_K).  Equal to ``ic_term`` in exact arithmetic."""
    kb = np.asarray(kb, dtype=np.float64)
    ds = float(delta_s(cosmo.a_init, a, cosmo))
    x = kb * C_OVER_H0 * T_NU0_EV / m_ev * ds
    P = np.asarray(sqrtPnu_init)
    return P * (I_func(x) - ds * cosmo.a_init * np.asarray(theta_over_delta_init) * nu_K(x))


def nu_response(kb, sqrtPcdm, a, cosmo: Cosmo, a_hist, sqrtPM_hist,
                sqrtPnu_init, theta_over_delta_init, sqrtPnu_prev=None,
                iters: int = 1, I_func=nu_I, epsrel=1e-11, nonempty=None, multipole=False):
    """Neutrino response per |k| bin (Eq. P-final, Sec. 4.3 (iii)-(iv), App. B).

    Inputs per bin b (arrays of length nb):
      kb            representative |k| of the bin [h/Mpc]
      sqrtPcdm      current P_cdm^{1/2}(k_b, a)
      a_hist        [n_hist] scale factors of the stored spectra (strictly
                    ascending, a_hist[0] >= a_i, a_hist[-1] < a)
      sqrtPM_hist   [n_hist, nb] stored P_M^{1/2}(k_b, a_j)
      sqrtPnu_init  [n_species, nb] P_nu,i^{1/2}(k_b)   (Eq. deltaI-nu)
      theta_over_delta_init [n_species, nb]  [theta_nu/delta_nu]_i(k_b)
      sqrtPnu_prev  [nb] P_nu^{1/2} of the previous step (None -> the
                    species-weighted IC value)
      multipole     initial-condition term by Eq. deltaI-multipole (j_1
                    integral, ic_term_multipole) instead of Eq. deltaI-nu
    The current node of P_M^{1/2} inside the integral is
      (1 - f_nu) P_cdm^{1/2}(a) + f_nu P_nu^{1/2}(guess),
    with the guess = sqrtPnu_prev for the first iteration (Sec. 4.3 (iii)) and
    the previous iteration's result afterwards (App. B).  Species results are
    weighted by Omega_nu,i / Omega_nu.

    Returns dict(R, sqrtPnu, sqrtPM) where R = P_nu^{1/2} / P_cdm^{1/2} (0 where
    P_cdm = 0) and sqrtPM = (1-f) P_cdm^{1/2} + f P_nu^{1/2} (App. B first
    equation).  With ``nonempty`` given, bins without modes return zeros.
    """
    kb = np.asarray(kb, dtype=np.float64)
    sqrtPcdm = np.asarray(sqrtPcdm, dtype=np.float64)
    nb = kb.size
    masses = np.asarray(cosmo.m_nu_ev, dtype=np.float64)
    wts = cosmo.species_weights()
    f = cosmo.f_nu
    if cosmo.omega_nu <= 0 or masses.size == 0 or masses.sum() <= 0:
        z = np.zeros(nb)
        return dict(R=z, sqrtPnu=z.copy(), sqrtPM=(1.0 - f) * sqrtPcdm)
    a_hist = np.asarray(a_hist, dtype=np.float64).reshape(-1)
    sqrtPM_hist = np.asarray(sqrtPM_hist, dtype=np.float64).reshape(a_hist.size, nb)
    Pi = np.asarray(sqrtPnu_init, dtype=np.float64).reshape(masses.size, nb)
    Ti = np.asarray(theta_over_delta_init, dtype=np.float64).reshape(masses.size, nb)
    if sqrtPnu_prev is None:
        guess = (wts[:, None] * Pi).sum(axis=0)
    else:
        guess = np.asarray(sqrtPnu_prev, dtype=np.float64)
    ic = np.zeros(nb)
    ic_fn = ic_term_multipole if multipole else ic_term
    for s, m in enumerate(masses):
        if m > 0:
            ic += wts[s] * ic_fn(kb, a, cosmo, m, Pi[s], Ti[s], I_func)
    if a < cosmo.a_init or (a_hist.size and (a_hist[0] < cosmo.a_init or a_hist[-1] >= a
                                              or np.any(np.diff(a_hist) <= 0))):
        raise ValueError("need a_i <= a_hist[0] < ... < a_hist[-1] < a")
    a_nodes = np.concatenate([a_hist, [a]])
    pnu = guess
    for _ in range(max(1, iters)):
        cur = (1.0 - f) * sqrtPcdm + f * pnu
        h_nodes = np.vstack([sqrtPM_hist, cur[None, :]]) if a_hist.size else cur[None, :]
        J = np.zeros(nb)
        for s, m in enumerate(masses):
            if m > 0:
                J += wts[s] * response_integral(kb, a, cosmo, m, a_nodes, h_nodes,
                                                I_func, epsrel)
        pnu = ic + J
    R = np.where(sqrtPcdm > 0, pnu / np.where(sqrtPcdm > 0, sqrtPcdm, 1.0), 0.0)
    pm = (1.0 - f) * sqrtPcdm + f * pnu
    if nonempty is not None:           # bins without modes carry no spectrum
        ne = np.asarray(nonempty, dtype=bool)
        R, pnu, pm = (np.where(ne, q, 0.0) for q in (R, pnu, pm))
    return dict(R=R, sqrtPnu=pnu, sqrtPM=pm)


# --------------------------------------------------------------------------
# Green's function, gradient, inverse transform, interpolation, kick
# (Eq. Poisson, Eq. phases, Sec. 4.3 (iv))
# --------------------------------------------------------------------------
def ratio_per_mode(kmag, kb, R, nonempty):
    """R(|k|): linear in ln k between non-empty bin representatives k_b,
    constant beyond the end bins (numpy.interp)."""
    ne = np.asarray(nonempty, dtype=bool)
    if not np.any(ne):
        return np.zeros_like(kmag)
    lk = np.log(np.where(kmag > 0, kmag, 1.0))
    return np.interp(lk, np.log(np.asarray(kb)[ne]), np.asarray(R)[ne])


def green_gradient(spec, box, a, cosmo: Cosmo, kb, R, nonempty, deconvolve=False):
    """Acceleration spectra acc_c(k) = -i k_c phi(k), c = x, y, z, with
    Poisson k^2 phi = -(3/2) Omega_M delta_M / a (Eq. Poisson, H0 = 1) and
    delta_M = delta_cdm [(1 - f_nu) + f_nu R(|k|)]  (Eq. phases with the
    total-matter sum of Sec. 4.3 (iv)).  k = 0 -> 0.  The gradient is the
    4-point finite difference of ``gradient_operator`` (zero on the Nyquist
    index).  Optional CIC deconvolution divides by prod_i sinc(k_i Delta/2)^4
    (assignment and interpolation windows).

    Pinned by: a single cosine density mode gives the analytic acceleration;
    point mass against the Ewald-summed periodic 1/r^2 force.
    """
    n = spec.shape[0]
    iz, iy, ix = mode_indices(n)
    phi = potential_spectrum(spec, box, a, cosmo, kb, R, nonempty, deconvolve)
    out = []
    for comp in (ix, iy, iz):
        out.append(-1j * gradient_operator(comp, n, box) * phi)
    return out   # [acc_x, acc_y, acc_z] spectra


def potential_spectrum(spec, box, a, cosmo: Cosmo, kb, R, nonempty, deconvolve=False, modes=None, ngrid=None):
    """phi(k) = G(k) delta_M(k) of ``green_gradient`` (Eq. Poisson with the
    neutrino-corrected delta_M), before the gradient.  By default over the
    whole half spectrum; with modes = (iz, iy, ix) and ngrid, at those modes
    (spec holding delta_k there).

    Pinned by (deconvolution): the divisor equals the square of the CIC
    assignment window measured from the oracle's own deposit and FFT (the
    single-particle DFT times e^{+ik.x}, averaged over sub-cell offsets)."""
    n = spec.shape[0] if modes is None else ngrid
    kf = 2.0 * math.pi / box
    iz, iy, ix = mode_indices(n) if modes is None else modes
    n2 = (iz * iz + iy * iy + ix * ix).astype(np.float64)
    kmag = kf * np.sqrt(n2)
    f = cosmo.f_nu
    Rm = ratio_per_mode(kmag, kb, R, nonempty) if f > 0 else np.zeros_like(kmag)
    fac = (1.0 - f) + f * Rm
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.where(n2 > 0, -1.5 * cosmo.omega_m / (a * kf * kf * np.where(n2 > 0, n2, 1.0)), 0.0)
    G = G * fac
    if deconvolve:
        def sinc(i):
            t = math.pi * i.astype(np.float64) / n
            return np.where(i == 0, 1.0, np.sin(t) / np.where(i == 0, 1.0, t))
        W = sinc(iz) * sinc(iy) * sinc(ix)
        G = G / W ** 4
    return G * spec


def gradient_operator(i, ngrid, box):
    """Fourier multiplier of the 4-point central finite-difference derivative
    d/dx f ~ [8 (f(x+D) - f(x-D)) - (f(x+2D) - f(x-2D))] / (12 D), D = L/N,
    on the periodic grid: i [8 sin(k D) - sin(2 k D)] / (6 D) with k D = 2 pi i / N.
    (The paper's code computes the PM force by finite differences of the mesh
    potential; it vanishes on the Nyquist index by construction.)"""
    t = 2.0 * math.pi * np.asarray(i, dtype=np.float64) / ngrid
    d = box / ngrid
    return (8.0 * np.sin(t) - np.sin(2.0 * t)) / (6.0 * d)


def inverse_fft(spec_c, ngrid):
    """Normalised inverse real 3-D DFT (numpy.fft.irfftn)."""
    return np.fft.irfftn(spec_c, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2))


def cic_interpolate(grid, c, w):
    """Trilinear (CIC) gather with the deposit's fixed-point weights / 2^48."""
    n = grid.shape[0]
    wx, wy, wz = (_corner_weights(w[0]), _corner_weights(w[1]), _corner_weights(w[2]))
    acc = np.zeros(c.shape[1])
    for dz in (0, 1):
        iz = (c[2] + dz) % n
        for dy in (0, 1):
            iy = (c[1] + dy) % n
            for dx in (0, 1):
                ix = (c[0] + dx) % n
                wt = (wx[dx] * wy[dy] * wz[dz]).astype(np.float64) / MASS_ONE
                acc += wt * grid[iz, iy, ix]
    return acc


@dataclass
class KickResult:
    F: np.ndarray
    bins: dict
    response: dict
    acc: np.ndarray          # [3, Np]
    vel: np.ndarray          # [3, Np] updated velocities
    extras: dict = field(default_factory=dict)


def pm_kick(c, w, vel, ngrid, box, a, kick, cosmo: Cosmo, n_kbins, a_hist, sqrtPM_hist,
            sqrtPnu_init, theta_over_delta_init, sqrtPnu_prev=None, iters=1,
            deconvolve=False, I_func=nu_I, epsrel=1e-11, keep_fields=False):
    """One PM long-range kick with Fourier-space neutrinos, steps (ii)-(iv) of
    Sec. 4.3 at one time step: deposit -> delta -> FFT -> P_cdm bins -> nu
    response (Eq. P-final) -> delta_M, Green, gradient -> inverse FFTs -> CIC
    interpolation -> u += acc * K."""
    npart = c.shape[1]
    F = cic_deposit(c, w, ngrid)
    delta = density_contrast(F, npart)
    spec = forward_fft(delta)
    bins = bin_power(spec, box, n_kbins)
    sqrtPcdm = np.sqrt(bins["P"])
    resp = nu_response(bins["k"], sqrtPcdm, a, cosmo, a_hist, sqrtPM_hist, sqrtPnu_init,
                       theta_over_delta_init, sqrtPnu_prev, iters, I_func, epsrel,
                       nonempty=bins["nonempty"])
    accs = green_gradient(spec, box, a, cosmo, bins["k"], resp["R"], bins["nonempty"],
                          deconvolve)
    acc = np.zeros((3, npart))
    fields = []
    for comp in range(3):
        g = inverse_fft(accs[comp], ngrid)
        if keep_fields:
            fields.append(g)
        acc[comp] = cic_interpolate(g, c, w)
    vnew = np.asarray(vel, dtype=np.float64) + acc * kick
    ex = dict(spec=spec, fields=fields) if keep_fields else {}
    return KickResult(F=F, bins=bins, response=resp, acc=acc, vel=vnew, extras=ex)


# --------------------------------------------------------------------------
# The step loop around the kick (Sec. 4.3: evolve the particles to the next
# time step, steps (ii)-(iv), store the total-matter spectrum, repeat)
# --------------------------------------------------------------------------
def drift_f64(x, u, ds, box):
    """FP64 positions moved by Delta x = u Delta s (u = a^2 dx/dt, ds = dt / a^2,
    Sec. 3.1), wrapped into [0, L): x' = x + (u * Delta s) as two IEEE FP64
    roundings (product, then sum; no fused multiply-add), then one add or
    subtract of L; a sum that rounds onto L itself becomes 0.
    Pinned by: a particle crossing either face wraps; the exact rational result
    within one rounding."""
    x = np.asarray(x, dtype=np.float64)
    xn = x + np.asarray(u, dtype=np.float64) * np.float64(ds)
    xn = np.where(xn < 0.0, xn + box, xn)
    xn = np.where(xn >= box, xn - box, xn)
    return np.where(xn >= box, 0.0, xn)


def drift_cell(cell, off, u, g, ngrid):
    """Int cell + FP32 offset positions moved by u Delta s, in FP32 with g =
    Delta s / Delta (cells per unit velocity) rounded to FP32 once:
      d = fl32(u g), o' = fl32(o + d), k = floor(o'), o'' = fl32(o' - k);
      o'' = 1 (a slightly negative o') becomes 0 with k + 1; cell = (cell + k) mod N.
    Each operation is one IEEE FP32 rounding (no fused multiply-add), so the
    cell decision is the same on every machine that follows it.
    Pinned by: the exact displacement within FP32 rounding; crossings of both
    faces; the o' -> 1 case."""
    u32 = np.asarray(u, dtype=np.float32)
    o = np.asarray(off, dtype=np.float32)
    d = u32 * np.float32(g)
    o1 = o + d
    k = np.floor(o1)
    o2 = o1 - k
    bump = o2 >= np.float32(1.0)
    o2 = np.where(bump, np.float32(0.0), o2).astype(np.float32)
    cn = np.mod(np.asarray(cell, dtype=np.int64) + k.astype(np.int64) + bump, ngrid)
    return cn, o2


@dataclass
class StepRun:
    """State of a run of steps: particles, velocities and the stored history.
    FP64 form: pos [3, Np] float64; FP32 form: (cell int64 [3, Np], off
    float32 [3, Np]), velocities kept as float32 values."""
    precision: str
    pos: object
    vel: np.ndarray
    a_hist: list
    hist: list               # rows P_M^{1/2}(k_b, a_j)
    prev: object = None      # P_nu^{1/2} of the last step (first-iteration guess)


def pm_step(run: StepRun, ngrid, box, a, kick, drift, cosmo: Cosmo, n_kbins, sqrtPnu_init,
            theta_over_delta_init, iters=1, I_func=nu_I, epsrel=1e-11):
    """One time step of Sec. 4.3: with the particles at a, steps (ii)-(iv)
    (deposit, P_cdm, neutrino response from the stored history with the last
    step's P_nu^{1/2} as the guess, Poisson, gradient, interpolation) and the
    kick u += acc * kick; then the total-matter row P_M^{1/2}(k_b, a) is stored
    and the particles move on by u * drift (drift = Delta s to the next step;
    0 after the last step).  Returns the KickResult of the step."""
    if run.precision == "fp64":
        c, w = quantise_positions_f64(run.pos, box, ngrid)
    else:
        c, w = quantise_positions_cell(run.pos[0], run.pos[1], ngrid)
    nh = len(run.a_hist)
    hist = np.asarray(run.hist, dtype=np.float64).reshape(nh, n_kbins)
    r = pm_kick(c, w, run.vel, ngrid, box, a, kick, cosmo, n_kbins, np.asarray(run.a_hist, dtype=np.float64),
                hist, sqrtPnu_init, theta_over_delta_init, sqrtPnu_prev=run.prev, iters=iters, I_func=I_func,
                epsrel=epsrel)
    run.vel = r.vel if run.precision == "fp64" else r.vel.astype(np.float32).astype(np.float64)
    run.a_hist.append(float(a))
    run.hist.append(r.response["sqrtPM"].copy())
    run.prev = r.response["sqrtPnu"].copy()
    if drift != 0.0:
        if run.precision == "fp64":
            run.pos = drift_f64(run.pos, run.vel, drift, box)
        else:
            run.pos = drift_cell(run.pos[0], run.pos[1], run.vel, np.float32(drift / (box / ngrid)), ngrid)
    return r


def leapfrog_factors(a_steps, cosmo):
    """Kick and drift factors of a leapfrog over the step epochs a_0 < ... < a_n:
    the kick at a_j spans the half steps around it, K(a_{j-1/2}, a_{j+1/2})
    with a_{j+1/2} = sqrt(a_j a_{j+1}) (half steps at the two ends), and the
    drift after it Delta s(a_j, a_{j+1}) (0 after the last)."""
    a = [float(v) for v in a_steps]
    mid = [math.sqrt(a[j] * a[j + 1]) for j in range(len(a) - 1)]
    lo = [a[0]] + mid
    hi = mid + [a[-1]]
    kicks = [kick_factor(l, h, cosmo) for l, h in zip(lo, hi)]
    drifts = [drift_factor(a[j], a[j + 1], cosmo) for j in range(len(a) - 1)] + [0.0]
    return kicks, drifts
