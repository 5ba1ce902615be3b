"""Seeded synthetic inputs for the PM kick (host side, untimed).

This module generates inputs only; it holds none of the kick's arithmetic and
imports neither the CUDA binding nor the oracle, so both can be fed the same
arrays.  The recipe stands in for the paper's CAMB transfer functions and
N-GenICs initial conditions (Sec. 4.3 (i), Sec. 4.4), which are not available:

* linear density field: Gaussian random field from a seeded PCG64 stream with
  the BBKS transfer function (Bardeen et al. 1986, shape Gamma = Omega_m h),
  primordial slope n_s, normalised to sigma_8 with a top-hat of 8 Mpc/h, grown
  with the LCDM growth factor D(a) (D(1) = 1);
* particles: one per lattice site q = (i + 1/2) L / n, moved by the
  Zel'dovich displacement x = q + D(a) psi(q), velocity u = a^2 H f D psi
  (u = a^2 dx/dt);
* stored spectra: P_M^{1/2}(k_b, a_j) = sqrt(P_lin(k_b^c)) D(a_j) at n_hist
  scale factors log-spaced on [a_i, a_kick), k_b^c the log-centre of bin b;
* neutrino initial conditions: P_nu,i^{1/2} = F(k/k_fs(a_i)) P_lin^{1/2}(k, a_i)
  with the matter-era response F(y) = 1/(1+y)^2 of App. A, and
  [theta/delta]_i = -a_i H(a_i) f(a_i) (linear growing mode, delta' + theta = 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
import scipy.fft as sfft
from scipy import integrate

T_NU0_EV = 1.68e-4
C_OVER_H0 = 2997.92458
ZETA3 = 1.2020569031595942


@dataclass(frozen=True)
class Workload:
    """One PM-kick workload.  ``precision`` is "fp64" (FP64 positions) or
    "fp32" (int32 cell + FP32 offset positions, FP32 grids)."""
    name: str
    ngrid: int
    npart_side: int
    box: float
    m_nu_total: float
    n_species: int = 3
    n_hist: int = 16
    n_kbins: int = 32
    precision: str = "fp64"
    a_init: float = 0.02
    a_kick: float = 0.1
    seed: int = 0
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    clustered: bool = False     # Zel'dovich at a = 1 (contention variant)
    m_species: tuple = ()       # unequal species masses [eV] (sum = m_nu_total); () = degenerate

    @property
    def npart(self) -> int:
        return self.npart_side ** 3

    @property
    def omega_nu(self) -> float:
        return self.m_nu_total / (93.14 * self.h * self.h)

    @property
    def omega_cdm(self) -> float:
        return self.omega_m - self.omega_nu

    @property
    def masses(self):
        if self.m_nu_total <= 0 or self.n_species <= 0:
            return ()
        if self.m_species:
            return tuple(float(m) for m in self.m_species)
        return tuple([self.m_nu_total / self.n_species] * self.n_species)


# The workloads of the benchmark configurations (plain FP64 kick; FP32 kick;
# precision form on a 1024^3 grid).  Batched and surrogate forms are built
# from these with ``replace``.
WORKLOADS = {
    "pm32_fp64": Workload("pm32_fp64", 32, 32, 256.0, 0.3, 3, 16, 32, "fp64"),
    "pm256_fp32_m015": Workload("pm256_fp32_m015", 256, 256, 512.0, 0.15, 3, 64, 128, "fp32"),
    "pm256_fp32_m030": Workload("pm256_fp32_m030", 256, 256, 512.0, 0.30, 3, 64, 128, "fp32"),
    "pm1024_p512_fp32": Workload("pm1024_p512_fp32", 1024, 512, 1000.0, 0.06, 3, 128, 256, "fp32"),
    "pm1024_p512_fp64": Workload("pm1024_p512_fp64", 1024, 512, 1000.0, 0.06, 3, 128, 256, "fp64"),
    # smaller analogue of the precision form (same cell size and particle:grid
    # ratio; every grid still larger than L2) for detailed profiling
    "pm512_p256_fp32": Workload("pm512_p256_fp32", 512, 256, 500.0, 0.06, 3, 128, 256, "fp32"),
    # surrogate form: 512^3 particles on a 512^3 grid (M_nu inside the surrogate's range)
    "pm512_p512_fp32": Workload("pm512_p512_fp32", 512, 512, 500.0, 0.3, 3, 128, 256, "fp32"),
}


def with_(w: Workload, **kw) -> Workload:
    return replace(w, **kw)


# Normal-hierarchy masses of the paper's S03NH run (Sec. 6.2, Table 1) [eV]
HIERARCHY_NH = (0.022, 0.024, 0.054)


def hierarchy(w: Workload, masses=HIERARCHY_NH) -> Workload:
    """w with unequal species masses (M_nu = their sum)."""
    return replace(w, m_nu_total=float(sum(masses)), n_species=len(masses), m_species=tuple(masses))


# ---------------------------------------------------------------- cosmology
def hubble(a, om):
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(om / a ** 3 + 1.0 - om)


def growth(a, om):
    """LCDM linear growth D(a) (D(1) = 1) and f = dlnD/dlna (Heath 1977)."""
    def I(x):
        v, _ = integrate.quad(lambda t: 1.0 / (t * float(hubble(t, om))) ** 3, 0.0, x,
                              epsabs=0.0, epsrel=1e-12, limit=200)
        return v
    i1 = I(1.0)
    ia = I(a)
    D = float(hubble(a, om)) * ia / i1
    f = -1.5 * om / (a ** 3 * float(hubble(a, om)) ** 2) + 1.0 / (a * a * float(hubble(a, om)) ** 3 * ia)
    return D, f


_GROWTH_TABLES = {}


def growth_interp(a, om):
    """D(a) from a 2048-point table in ln a on [0.005, 2] (linear in ln a;
    relative error < 1e-7), for drawing many scenarios quickly."""
    tab = _GROWTH_TABLES.get(om)
    if tab is None:
        la = np.linspace(math.log(0.005), math.log(2.0), 2048)
        tab = (la, np.array([growth(math.exp(x), om)[0] for x in la]))
        _GROWTH_TABLES[om] = tab
    return np.interp(np.log(np.asarray(a, dtype=np.float64)), tab[0], tab[1])


def bbks_power_unnormed(k, om, h, n_s):
    k = np.asarray(k, dtype=np.float64)
    q = k / (om * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        T = np.log1p(2.34 * q) / (2.34 * q) * (
            1 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
    T = np.where(k > 0, T, 1.0)
    return np.where(k > 0, k ** n_s * T * T, 0.0)


def power_norm(om, h, n_s, sigma8):
    def integrand(lnk):
        k = math.exp(lnk)
        x = 8.0 * k
        W = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3
        return k ** 3 * float(bbks_power_unnormed(k, om, h, n_s)) * W * W / (2 * math.pi ** 2)
    s2, _ = integrate.quad(integrand, math.log(1e-5), math.log(1e2), limit=500, epsrel=1e-10)
    return sigma8 ** 2 / s2


def linear_power(k, w: Workload):
    """Linear P(k) at a = 1 in (Mpc/h)^3."""
    return power_norm(w.omega_m, w.h, w.n_s, w.sigma8) * bbks_power_unnormed(
        k, w.omega_m, w.h, w.n_s)


# ---------------------------------------------------------------- particles
def displacement_field(w: Workload):
    """Zel'dovich displacement psi(q) at D = 1 on the particle lattice, [3, n^3]."""
    n = w.npart_side
    rng = np.random.Generator(np.random.PCG64(w.seed))
    white = rng.standard_normal((n, n, n))
    wk = sfft.rfftn(white, workers=-1)
    del white
    kf = 2 * math.pi / w.box
    f = np.fft.fftfreq(n, d=1.0 / n)
    kz = (f * kf)[:, None, None]
    ky = (f * kf)[None, :, None]
    kx = (np.arange(n // 2 + 1) * kf)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    amp = np.sqrt(linear_power(np.sqrt(k2), w) * n ** 3 / w.box ** 3)
    dk = wk * amp
    del wk, amp
    dk[0, 0, 0] = 0
    nyq = n // 2
    psi = np.empty((3, n * n * n))
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    for comp, kc in enumerate((kx, ky, kz)):
        g = 1j * kc * dk * inv_k2
        # keep the field real-symmetric: drop the Nyquist planes
        g[nyq, :, :] = 0
        g[:, nyq, :] = 0
        g[:, :, nyq] = 0
        psi[comp] = sfft.irfftn(g, s=(n, n, n), workers=-1).reshape(-1)
    return psi


def particles(w: Workload, a=None):
    """Zel'dovich particles at scale factor ``a`` (default a_kick).

    Returns dict(pos64 [3,Np] float64 in [0, L), vel [3,Np] float64)."""
    a = w.a_kick if a is None else a
    n = w.npart_side
    psi = displacement_field(w)
    a_pos = 1.0 if w.clustered else a
    D, f = growth(a_pos, w.omega_m)
    Dv, fv = growth(a, w.omega_m)
    i = (np.arange(n, dtype=np.float64) + 0.5) * (w.box / n)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    q = np.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)])
    pos = np.mod(q + D * psi, w.box)
    pos = np.where(pos >= w.box, 0.0, pos)
    vel = (a * a * float(hubble(a, w.omega_m)) * fv * Dv) * psi
    return dict(pos64=pos, vel=vel)


def to_cell_offset(pos64, box, ngrid):
    """FP64 positions -> packed int32 [6, Np]: rows 0-2 cell index, rows 3-5 the
    FP32 offset in [0, 1) (bit pattern stored in int32)."""
    u = np.asarray(pos64, dtype=np.float64) / (box / ngrid)
    c = np.floor(u)
    off = (u - c).astype(np.float32)
    bump = off >= np.float32(1.0)
    off = np.where(bump, np.float32(0.0), off)
    c = np.mod(c.astype(np.int64) + bump, ngrid).astype(np.int32)
    out = np.empty((6, c.shape[1]), dtype=np.int32)
    out[:3] = c
    out[3:] = off.view(np.int32)
    return out


def split_cell_offset(packed):
    packed = np.ascontiguousarray(packed)
    return packed[:3].astype(np.int64), packed[3:].copy().view(np.float32)


# ---------------------------------------------------------------- tables
def bin_log_centres(w: Workload):
    kmin = 2 * math.pi / w.box
    kmax = math.sqrt(3.0) * math.pi * w.ngrid / w.box
    b = np.arange(w.n_kbins) + 0.5
    return kmin * (kmax / kmin) ** (b / w.n_kbins)


def history(w: Workload):
    """Stored spectra: a_hist [n_hist], sqrtPM_hist [n_hist, n_kbins]."""
    j = np.arange(w.n_hist, dtype=np.float64)
    a_hist = w.a_init * (w.a_kick / w.a_init) ** (j / max(w.n_hist, 1))
    kc = bin_log_centres(w)
    p = np.sqrt(linear_power(kc, w))
    D = np.array([growth(a, w.omega_m)[0] for a in a_hist])
    return a_hist, D[:, None] * p[None, :]


def nu_initial(w: Workload):
    """sqrtPnu_init [n_species, n_kbins], theta_over_delta_init [n_species, n_kbins]."""
    return nu_initial_at(bin_log_centres(w), w)


def nu_initial_at(kc, w: Workload):
    """The neutrino initial conditions of ``nu_initial`` at wavenumbers kc."""
    kc = np.asarray(kc, dtype=np.float64)
    ai = w.a_init
    D, f = growth(ai, w.omega_m)
    H = float(hubble(ai, w.omega_m))
    om_a = w.omega_m / ai ** 3 / H ** 2
    p = np.sqrt(linear_power(kc, w)) * D
    ns = len(w.masses)
    P = np.zeros((max(ns, 1), kc.size))
    T = np.zeros((max(ns, 1), kc.size))
    for s, m in enumerate(w.masses):
        v2 = 2 * math.log(2) / (3 * ZETA3) * (m * ai / T_NU0_EV) ** 2
        kfs = math.sqrt(1.5 * om_a * v2) * ai * H / C_OVER_H0
        P[s] = p / (1.0 + kc / kfs) ** 2
        T[s] = -ai * H * f
    return P, T


# ---------------------------------------------------------------- surrogate training scenarios
SURROGATE_K = (0.002, 20.0)          # h/Mpc range of the training bins
SURROGATE_M_NU = (0.04, 0.65)        # eV, a little beyond the surrogate's [0.05, 0.6]
SURROGATE_A = (0.04, 1.0)


def surrogate_kbins(n_kbins: int = 256):
    """Log-spaced wavenumbers of the training bins [h/Mpc]."""
    lo, hi = SURROGATE_K
    return lo * (hi / lo) ** ((np.arange(n_kbins) + 0.5) / n_kbins)


def surrogate_group(seed: int, n_scen: int, n_kbins: int = 256, n_hist_max: int = 128):
    """One neutrino mass and n_scen seeded scenarios of (a, stored history,
    current CDM amplitude) on the surrogate's k bins.  Histories follow
    sqrt(P_lin(k)) D(a') times a smooth perturbation 1 + eps(k) sin(pi v),
    v = (ln a' - ln a_i)/(ln a - ln a_i) in [0, 1) (vanishing at a_i), eps(k) =
    e0 + e1 tanh(ln(k / 0.1 h/Mpc)), e0, e1 uniform in [-0.08, 0.08]; node counts
    from {4, 8, 16, 32, 64, 128} (<= n_hist_max), log-spaced on [a_i, a); the
    current amplitude is sqrt(P_lin) D(a) (1 + 0.02 N(0, 1)).
    Returns (workload carrying M_nu, kb, list of scenario dicts)."""
    rng = np.random.default_rng(10_000 + seed)
    m_nu = float(rng.uniform(*SURROGATE_M_NU))
    w = Workload(f"sur{seed}", 32, 32, 1000.0, m_nu, 3, 16, n_kbins, "fp64")
    kb = surrogate_kbins(n_kbins)
    p = np.sqrt(linear_power(kb, w))
    scen = []
    choices = [n for n in (4, 8, 16, 32, 64, 128) if n <= n_hist_max]
    for _ in range(n_scen):
        a = float(math.exp(rng.uniform(math.log(SURROGATE_A[0]), math.log(SURROGATE_A[1]))))
        nh = int(rng.choice(choices))
        j = np.arange(nh, dtype=np.float64)
        a_hist = w.a_init * (a / w.a_init) ** (j / nh)
        v = (np.log(a_hist) - math.log(w.a_init)) / (math.log(a) - math.log(w.a_init))
        e0, e1 = rng.uniform(-0.08, 0.08, size=2)
        eps = e0 + e1 * np.tanh(np.log(kb / 0.1))
        D = growth_interp(a_hist, w.omega_m)
        hist = D[:, None] * p[None, :] * (1.0 + eps[None, :] * np.sin(np.pi * v)[:, None])
        cur = p * float(growth_interp(a, w.omega_m)) * (1.0 + 0.02 * rng.normal(size=n_kbins))
        scen.append(dict(a=a, a_hist=a_hist, hist=hist, sqrtPcdm=cur))
    return w, kb, scen


# ---------------------------------------------------------------- batched form
BATCH_GRIDS = (64, 128, 192)
BATCH_M_NU = (0.0, 0.06, 0.15, 0.3, 0.6)


def batched_boxes(n_boxes: int = 32, n_hist: int = 32, n_kbins: int = 64):
    """The batched configuration: box b (seed b) has grid BATCH_GRIDS[b % 3]
    with one particle per cell, side L = 200 + 300 b / 31 Mpc/h and
    M_nu = BATCH_M_NU[b % 5]; FP32 form."""
    out = []
    for b in range(n_boxes):
        n = BATCH_GRIDS[b % 3]
        L = 200.0 + 300.0 * b / 31.0
        out.append(Workload(f"box{b}", n, n, L, BATCH_M_NU[b % 5], 3, n_hist, n_kbins, "fp32", seed=b))
    return out
