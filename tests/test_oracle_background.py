"""Pins of the oracle's Sec. 4.4 background: the energy density of massive
neutrinos from Eq. relativistic (relativistic Fermi-Dirac momenta with
eps = sqrt(m^2 + q^2/a^2)) and radiation in H(a), against the textbook
limits of a relativistic and a non-relativistic Fermi gas, adaptive
quadrature, and closed forms of s(a) in radiation and matter domination."""
import math

import numpy as np
from scipy import integrate, special

from oracle import pm_oracle as O

Z3, Z5 = float(special.zeta(3)), float(special.zeta(5))


def test_energy_ratio_against_adaptive_quadrature():
    for y in (0.05, 0.3, 1.0, 3.0, 30.0):
        q, _ = integrate.quad(lambda x: math.sqrt(1 + (x / y) ** 2) * x * x / (math.exp(x) + 1), 0, 200,
                              points=[y], limit=500, epsabs=0, epsrel=1e-13)
        assert abs(float(O.nu_energy_ratio(y)) / (q / (1.5 * Z3)) - 1) < 1e-12


def test_energy_ratio_non_relativistic_limit():
    # eps = m + q^2 / (2 m a^2) + ...: R = 1 + <x^2> / (2 y^2), <x^2> = 15 zeta(5) / zeta(3)
    for y in (1e3, 1e4):
        R = float(O.nu_energy_ratio(y))
        assert abs((R - 1) * 2 * y * y / (15 * Z5 / Z3) - 1) < 3e-4 * (1e3 / y) ** 2


def test_massless_limit_is_the_relativistic_fermi_gas():
    # m -> 0: rho = m n R(m / T) with n = 3 zeta(3) T^3 / (2 pi^2) per species
    # (g = 2) must equal (7/8)(pi^2/15) T^4, i.e. 7/8 (4/11)^{4/3} of the photon
    # density at T_gamma = (11/4)^{1/3} T_nu
    T = O.T_NU0_EV
    for m in (1e-9, 1e-7):
        n = 3 * Z3 * T ** 3 / (2 * math.pi ** 2)
        rho = m * n * float(O.nu_energy_ratio(m / T))
        assert abs(rho / (7 / 8 * math.pi ** 2 / 15 * T ** 4) - 1) < 1e-6
        rho_gamma = math.pi ** 2 / 15 * ((11 / 4) ** (1 / 3) * T) ** 4
        assert abs(rho / rho_gamma / O.NU_TO_GAMMA - 1) < 1e-6


def _cosmo(m=(0.1, 0.1, 0.1), h=0.7, om=0.3):
    onu = sum(m) / (93.14 * h * h)
    return O.Cosmo(om - onu, onu, h, m, 0.02, relativistic=True)


def test_background_is_flat_and_reduces_at_late_times():
    c = _cosmo()
    assert abs(float(O.hubble(1.0, c)) - 1) < 1e-15
    # heavy neutrinos (10 eV: non-relativistic for a >> 1e-5) and no radiation
    # at a = 0.5 would be the matter + Lambda background; the radiation and the
    # residual kinetic energy shift it by Omega_r (a^-4 - 1) + O(1e-6)
    heavy = _cosmo(m=(10.0,))
    a = 0.5
    e2 = float(heavy.e2(a))
    om, orad = heavy.omega_m, heavy.omega_r
    want = om / a ** 3 + (1 - om) + orad * (a ** -4 - 1)
    assert abs(e2 / want - 1) < 1e-6
    # without massive neutrinos the radiation holds three massless species
    cdm = O.Cosmo(0.3, 0.0, 0.7, (), 0.02, relativistic=True)
    assert abs(cdm.omega_r / (O.OMEGA_GAMMA_H2 / 0.49) - (1 + 3 * O.NU_TO_GAMMA)) < 1e-15


def test_radiation_era_superconformal_time():
    # a ~ 1e-9: radiation dominates (matter / radiation ~ 1e-5), H = sqrt(Om_rad) a^-2,
    # so s(a1) - s(a0) = ln(a1 / a0) / sqrt(Om_rad); the massive species count
    # as radiation there: Om_nu,i R(m a/T) a^-3 -> Om_nu,i (7 pi^4/(180 zeta 3)) (T/m) a^-4
    c = _cosmo()
    C = 7 * math.pi ** 4 / (180 * Z3)
    orad = c.omega_r + sum(c.omega_nu * w * C * O.T_NU0_EV / m for m, w in zip(c.m_nu_ev, c.species_weights()))
    a0, a1 = 1e-10, 1e-9
    ds = float(O.delta_s(a0, a1, c))
    assert abs(ds * math.sqrt(orad) / math.log(a1 / a0) - 1) < 2e-4
    # and the non-relativistic background is the same call without the flag
    nr = O.Cosmo(c.omega_cdm, c.omega_nu, c.h, c.m_nu_ev, c.a_init)
    assert float(O.delta_s(0.05, 0.1, nr)) == float(O.delta_s(0.05, 0.1, nr.omega_m))


def test_kick_and_drift_factors_follow_the_background():
    # at a ~ 1 radiation is negligible: the factors agree with matter + Lambda to ~1e-4
    c = _cosmo()
    nr = O.Cosmo(c.omega_cdm, c.omega_nu, c.h, c.m_nu_ev, c.a_init)
    k_rel, k_nr = O.kick_factor(0.5, 0.6, c), O.kick_factor(0.5, 0.6, nr)
    assert 0 < abs(k_rel / k_nr - 1) < 1e-3
    # early on, radiation and relativistic neutrinos raise H, so K = int da / (a H) is smaller
    assert O.kick_factor(0.02, 0.03, c) < O.kick_factor(0.02, 0.03, nr)
