"""Pins of the oracle's free-streaming kernel I(x) (Eq. I.def, App. C) and
background helpers against values the paper and the mathematics fix."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import pm_oracle as O

ZETA3 = 1.2020569031595942854
ZETA5 = 1.0369277551433699263


def test_I_at_zero_is_one():
    # Eq. I.def is normalised so that I(0) = 1 (Sec. 3.2).
    assert abs(O.nu_I(0.0) - 1.0) < 1e-14


def test_I_small_x_slope():
    # App. C: I(x) ~ 1 - 5 zeta(5) / (2 zeta(3)) x^2 = 1 - 2.1566 x^2.
    # (1 - I)/x^2 = c1 - c2 x^2 + ...: Richardson-extrapolate c1 from two x.
    x1, x2 = 2e-3, 4e-3
    s1 = (1.0 - O.nu_I(x1)) / x1 ** 2
    s2 = (1.0 - O.nu_I(x2)) / x2 ** 2
    c1 = (s1 * x2 ** 2 - s2 * x1 ** 2) / (x2 ** 2 - x1 ** 2)
    assert abs(c1 - 5 * ZETA5 / (2 * ZETA3)) < 1e-6
    assert abs(5 * ZETA5 / (2 * ZETA3) - 2.1566) < 1e-4   # printed value


def test_I_large_x_limit():
    # App. C: I(x) ~ 1 / (3 zeta(3) x^4) = 0.2773 / x^4.
    vals = [O.nu_I(x) * x ** 4 for x in (300.0, 1000.0)]
    assert abs(vals[-1] - 1.0 / (3 * ZETA3)) < 1e-5
    assert abs(1.0 / (3 * ZETA3) - 0.2773) < 1e-4          # printed value
    # approach from one side, monotone in x
    assert abs(vals[0] - 1 / (3 * ZETA3)) > abs(vals[1] - 1 / (3 * ZETA3))


def test_I_against_brute_force_partial_sums():
    # Direct partial sums of the App. C series with 2e6 terms; the mean of two
    # consecutive partial sums of an alternating series with terms ~ n^-3 is
    # accurate to ~ n^-4 ~ 1e-25.
    n = np.arange(1, 2_000_002, dtype=np.float64)
    sign = np.where(n % 2 == 1, 1.0, -1.0)
    for x in (0.3, 1.0, 3.0, 10.0, 40.0):
        t = sign * n / (n * n + x * x) ** 2
        s_a = t[:-1].sum()
        s_b = s_a + t[-1]
        ref = 0.5 * (s_a + s_b) * 4.0 / (3.0 * ZETA3)
        assert abs(O.nu_I(x) - ref) <= 1e-12 * max(ref, 1e-30) + 1e-16


def test_I_against_quadrature_of_definition():
    # Eq. I.def with f0 ~ 1/(e^q + 1): I(x) = int j0(q x) q^2 f0 / int q^2 f0,
    # int q^2 f0 dq = 3 zeta(3) / 2; j0(qx) q^2 = q sin(qx) / x.
    # Evaluated with QUADPACK's oscillatory-weight routine (weight='sin').
    for x in (0.1, 0.5, 1.0, 2.0, 5.0, 10.0):
        # q e^-q / (1 + e^-q) is below 1e-30 beyond q = 80
        num, _ = integrate.quad(lambda q: q * math.exp(-q) / (1.0 + math.exp(-q)), 0.0, 80.0,
                                weight="sin", wvar=x, epsabs=1e-16, epsrel=1e-13, limit=400)
        ref = num / x / (1.5 * ZETA3)
        assert abs(O.nu_I(x) - ref) < 1e-10 * max(1.0, abs(ref)) + 1e-13


def test_integral_of_x_I():
    # Sec. 3.3.2: delta_hdm(k >> k_fs) ~ -(m a)^2 phi int X I(X) dX equals
    # -<v^-2> phi (Eq. small-scales) with Eq. v2, which requires
    # int_0^inf x I(x) dx = 2 ln 2 / (3 zeta 3) = 0.38442283...
    X = 400.0
    xs = np.concatenate([np.linspace(0, 4, 4001)[:-1], np.geomspace(4, X, 6001)])
    f = xs * O.nu_I(xs)
    body = integrate.simpson(f, x=xs)
    tail = 1.0 / (3 * ZETA3) / (2 * X * X)
    assert abs(body + tail - 2 * math.log(2) / (3 * ZETA3)) < 2e-8


def test_fit_accuracy_as_printed():
    # App. C: |Delta I| <~ 0.07% absolute for all x; relative <~ 1% on [0, 2].
    x = np.concatenate([np.linspace(0, 2, 2001), np.geomspace(2, 200, 2000)])
    ex = O.nu_I(x)
    fit = O.nu_I_fit(x)
    assert np.max(np.abs(fit - ex)) < 7.5e-4
    sel = x <= 2
    assert np.max(np.abs(fit[sel] / ex[sel] - 1)) < 1.2e-2


def test_f_nu_printed():
    # Sec. 2.1: f_nu ~ 0.022 (0.147 / Omega_M h^2)(M_nu / 0.3 eV).
    om, h = 0.3, 0.7
    f = O.omega_nu_from_mass(0.3, h) / om
    assert abs(f - 0.022 * 0.147 / (om * h * h)) < 3e-4


def test_kfs_and_velocity_printed():
    # Eq. kfs: k_fs ~ 0.08 / sqrt(1+z) sqrt(Om/0.3) (m / 0.1 eV) h/Mpc at z = 0.
    k = O.free_streaming_k(1.0, 0.1, 0.3)
    assert abs(k / 0.08 - 1) < 0.05
    # Eq. v2: <v^-2>^{-1/2} ~ 810 km/s (1+z) (0.1 eV / m).
    v = 299792.458 * O.T_NU0_EV / 0.1 * math.sqrt(3 * ZETA3 / (2 * math.log(2)))
    assert abs(v / 810 - 1) < 0.01


def test_delta_s_and_kick_closed_forms():
    # Einstein-de Sitter (Omega_M = 1): s = 2 (a0^-1/2 - a1^-1/2),
    # K = int da/(aH) = (2/3)(a1^{3/2} - a0^{3/2}).
    for a0, a1 in ((0.02, 0.1), (0.1, 0.1001), (0.3, 1.0)):
        assert abs(O.delta_s(a0, a1, 1.0) - 2 * (a0 ** -0.5 - a1 ** -0.5)) < 1e-13 * a1 ** -0.5 * 10
        assert abs(O.kick_factor(a0, a1, 1.0) - 2 / 3 * (a1 ** 1.5 - a0 ** 1.5)) < 1e-14
        assert abs(O.drift_factor(a0, a1, 1.0) - 2 * (a0 ** -0.5 - a1 ** -0.5)) < 1e-12


def test_delta_s_against_adaptive_quad_lcdm():
    om = 0.3
    for a0, a1 in ((0.02, 0.1), (0.02, 1.0)):
        ref, _ = integrate.quad(lambda a: 1 / (a ** 3 * math.sqrt(om / a ** 3 + 1 - om)), a0, a1,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert abs(O.delta_s(a0, a1, om) - ref) <= 3e-13 * abs(ref)


def test_delta_s_short_interval_high_precision():
    # s - s' for a' -> a must not lose digits (it multiplies I in Eq. P-final).
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    om = 0.3
    a0, a1 = 0.5, 0.5000001
    ref = mpmath.quad(lambda a: 1 / (a ** 3 * mpmath.sqrt(om / a ** 3 + 1 - om)),
                      [mpmath.mpf(a0), mpmath.mpf(a1)])
    assert abs(O.delta_s(a0, a1, om) / float(ref) - 1) < 1e-14


def test_l1_multipole_kernel_equals_I():
    # Eq. deltaI-multipole with delta f_1 = f_0' m a_i theta / k (Sec. 4.1): the
    # l = 1 momentum integral of j_1 equals -a_i theta (s - s_i) I(y) exactly
    # (d/dz [z^2 j_1(z)] = z^2 j_0(z)); K from the j_1 integral against I from
    # the App. C series, and K's own small-y limit
    from scipy import special as sp
    y = np.array([1e-2, 0.1, 0.5, 0.99, 1.0, 2.0, 5.0, 20.0, 100.0])
    K = O.nu_K(y)
    I = O.nu_I(y)
    assert np.allclose(K, I, rtol=1e-9, atol=1e-15)
    c2 = 5 * sp.zeta(5) / (2 * sp.zeta(3))
    for yy in (1e-4, 1e-3):
        assert abs(float(O.nu_K(yy)) - (1 - c2 * yy * yy)) < 1e-9
    assert float(O.nu_K(0.0)) == 1.0


def test_multipole_ic_term_in_the_response():
    # the response with the j_1 form of the initial-condition term equals the
    # integrated-by-parts form (Eq. deltaI-nu)
    m = 0.1
    c = O.Cosmo(0.3 - 3 * m / (93.14 * 0.49), 3 * m / (93.14 * 0.49), 0.7, (m, m, m), 0.02)
    kb = np.geomspace(0.005, 0.5, 5)
    pi = np.tile(10.0 / (1 + kb / 0.05) ** 2, (3, 1))
    ti = np.full((3, 5), -0.3)
    cur = 20.0 / (1 + kb / 0.2)
    r0 = O.nu_response(kb, cur, 0.05, c, [], np.zeros((0, 5)), pi, ti)
    r1 = O.nu_response(kb, cur, 0.05, c, [], np.zeros((0, 5)), pi, ti, multipole=True)
    assert np.allclose(r1["R"], r0["R"], rtol=1e-9, atol=0)
