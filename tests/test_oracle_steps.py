"""Pins of the oracle's step loop (Sec. 4.3: evolve the particles, steps
(ii)-(iv), store P_M, repeat): the drift against exact rational arithmetic,
and the growth of a single small-amplitude mode through many steps against
the linear growth factor, without neutrinos and with heavy neutrinos (which
cluster like CDM on the box scale, Sec. 3.3.2) -- a run that lost the stored
history would miss the integral term of Eq. P-final and grow too slowly."""
import math
from fractions import Fraction

import numpy as np

from oracle import pm_oracle as O


def test_drift_f64_exact_and_wrapping():
    rng = np.random.default_rng(5)
    L = 100.0
    x = rng.uniform(0, L, 2000)
    u = rng.normal(0, 30, 2000)
    ds = 0.37
    xn = O.drift_f64(x[None], u[None], ds, L)[0]
    for xi, ui, yi in zip(x, u, xn):
        exact = Fraction(xi) + Fraction(float(np.float64(ui) * np.float64(ds)))
        exact = exact % Fraction(L)
        assert 0 <= yi < L
        d = abs(Fraction(yi) - exact)
        d = min(d, Fraction(L) - d)                   # periodic distance
        assert d <= Fraction(2.0 ** -52) * L * 2
    # crossings of both faces
    y = O.drift_f64(np.array([[99.5, 0.5]]), np.array([[2.0, -2.0]]), 1.0, L)[0]
    assert np.allclose(y, [1.5, 98.5], atol=1e-13, rtol=0)


def test_drift_cell_fp32_rules():
    n = 16
    rng = np.random.default_rng(7)
    cell = rng.integers(0, n, (3, 4000))
    off = rng.uniform(0, 1, (3, 4000)).astype(np.float32)
    u = rng.normal(0, 3, (3, 4000)).astype(np.float32)
    g = np.float32(0.731)
    cn, on = O.drift_cell(cell, off, u, g, n)
    assert on.dtype == np.float32 and np.all(on >= 0) and np.all(on < 1)
    assert np.all((cn >= 0) & (cn < n))
    # the position moved by u g cells to within FP32 rounding of the offset sums
    before = cell + off.astype(np.float64)
    after = cn + on.astype(np.float64)
    dd = np.mod(after - before - u.astype(np.float64) * float(g) + n / 2, n) - n / 2
    assert np.max(np.abs(dd)) < 4 * 2.0 ** -24 * (1 + np.abs(u).max() * float(g))
    # o' slightly below zero: o' - floor(o') rounds to 1 -> offset 0, same cell
    c1, o1 = O.drift_cell(np.array([[5]]), np.array([[0.0]], np.float32), np.array([[-2.0 ** -30]], np.float32),
                          np.float32(1.0), n)
    assert c1[0, 0] == 5 and o1[0, 0] == 0.0
    # a crossing of the lower face wraps the cell
    c2, o2 = O.drift_cell(np.array([[0]]), np.array([[0.25]], np.float32), np.array([[-0.5]], np.float32),
                          np.float32(1.0), n)
    assert c2[0, 0] == n - 1 and o2[0, 0] == np.float32(0.75)


def lcdm_growth(a, om):
    from scipy import integrate
    H = lambda t: math.sqrt(om / t ** 3 + 1 - om)
    I = lambda x: integrate.quad(lambda t: 1.0 / (t * H(t)) ** 3, 0, x, epsrel=1e-12)[0]
    Ia = I(a)
    return H(a) * Ia, -1.5 * om / (a ** 3 * H(a) ** 2) + 1.0 / (a * a * H(a) ** 3 * Ia)


def single_mode_run(cos, n=32, L=256.0, ai=0.02, af=0.1, nsteps=40, nk=8):
    """A single sine mode of 1% amplitude at a_i, grown by pm_step through
    nsteps leapfrog steps log-spaced in a; returns (measured growth,
    D(af)/D(ai), the run)."""
    om = cos.omega_m
    k0 = 2 * math.pi / L
    amp = 0.01 / k0
    q1 = (np.arange(n) + 0.5) * L / n
    qz, qy, qx = np.meshgrid(q1, q1, q1, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()])
    psi = np.zeros_like(q)
    psi[0] = amp * np.sin(k0 * q[0])
    Di, fi = lcdm_growth(ai, om)
    Df, _ = lcdm_growth(af, om)
    H = math.sqrt(om / ai ** 3 + 1 - om)
    run = O.StepRun("fp64", np.mod(q + psi, L), ai * ai * H * fi * psi, [], [])
    # neutrino ICs: fully clustered (P_nu,i = P_cdm,i, measured) on the growing mode
    ns = max(len(cos.m_nu_ev), 1)
    c0, w0 = O.quantise_positions_f64(run.pos, L, n)
    b0 = O.bin_power(O.forward_fft(O.density_contrast(O.cic_deposit(c0, w0, n), n ** 3)), L, nk)
    pi = np.tile(np.sqrt(b0["P"]), (ns, 1))
    ti = np.full((ns, nk), -ai * H * fi)
    a_steps = np.exp(np.linspace(math.log(ai), math.log(af), nsteps + 1))
    kicks, drifts = O.leapfrog_factors(a_steps, cos)
    for a, K, S in zip(a_steps, kicks, drifts):
        O.pm_step(run, n, L, a, K, S, cos, nk, pi, ti, epsrel=1e-8)
    disp = run.pos[0] - q[0]
    disp = (disp + L / 2) % L - L / 2
    fit = (disp * np.sin(k0 * q[0])).sum() / (np.sin(k0 * q[0]) ** 2).sum()
    return fit / amp, Df / Di, run, q


def test_single_mode_linear_growth_cdm_only():
    cos = O.Cosmo(0.3, 0.0, 0.7, (), 0.02)
    growth, want, run, q = single_mode_run(cos)
    assert abs(growth / want - 1) < 0.01
    assert np.max(np.abs(run.pos[1] - q[1])) < 1e-9 and np.max(np.abs(run.pos[2] - q[2])) < 1e-9
    assert len(run.a_hist) == 41 and np.all(np.diff(run.a_hist) > 0)


def test_single_mode_growth_with_heavy_neutrinos_uses_the_history():
    # 3 x 3 eV: f_nu ~ 0.66, k_fs >> k of the mode, so the neutrinos follow
    # the CDM and the total matter grows as D(a) with Omega_M = 0.3
    m = (3.0, 3.0, 3.0)
    onu = sum(m) / (93.14 * 0.49)
    cos = O.Cosmo(0.3 - onu, onu, 0.7, m, 0.02)
    assert cos.f_nu > 0.6
    growth, want, run, _ = single_mode_run(cos, nsteps=24)
    assert abs(growth / want - 1) < 0.01, growth / want
    # the stored rows grow with the mode: P_M^{1/2}(k_0) ~ D(a)
    h = np.array(run.hist)[:, 0]
    assert abs(h[-1] / h[0] / want - 1) < 0.02
