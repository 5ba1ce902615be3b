"""Pins of the oracle's neutrino response (Eq. P-final, Eq. deltaI-nu,
Sec. 3.3, App. A, App. B) against closed forms, an independent quadrature
and the paper's limits."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import pm_oracle as O

ONE = lambda x: np.ones_like(np.asarray(x, dtype=float))   # I == 1 (heavy-nu limit)


def eds(m=0.1, ai=0.01, eps=1e-8):
    """Einstein-de Sitter (Omega_M = 1) with a negligible neutrino fraction."""
    return O.Cosmo(omega_cdm=1.0 - eps, omega_nu=eps, h=0.7, m_nu_ev=(m,), a_init=ai)


def test_ic_term_closed_form_eds():
    # I == 1, EdS, growing mode [theta/delta]_i = -a_i H_i f_i = -a_i^{-1/2}:
    # the IC piece of Eq. P-final is P_i (3 - 2 sqrt(a_i / a)).
    ai, a = 0.01, 0.2
    c = eds(ai=ai)
    got = O.ic_term(np.array([0.3]), a, c, 0.1, np.array([2.0]), np.array([-ai ** -0.5]), ONE)
    assert abs(got[0] - 2.0 * (3 - 2 * math.sqrt(ai / a))) < 1e-13


def test_integral_term_constant_history_closed_form():
    # I == 1, EdS, P_M^{1/2} == c: J = 1.5 c int 2 (a'^-1/2 - a^-1/2) a'^-1/2 da'
    #   = 3 c [ln(a/a_i) - 2 (1 - sqrt(a_i/a))].
    ai, a, cval = 0.01, 0.3, 1.7
    c = eds(ai=ai)
    J = O.response_integral(np.array([0.1, 2.0]), a, c, 0.1, [ai, a],
                            np.array([[cval, cval], [cval, cval]]), ONE)
    ref = 3 * cval * (math.log(a / ai) - 2 * (1 - math.sqrt(ai / a)))
    assert np.allclose(J, ref, rtol=1e-10, atol=0)


def test_fluid_limit_growing_mode():
    # Sec. 3.3.1: with I == 1 the response is the pressureless-fluid solution.
    # A growing mode P^{1/2} = h0 a / a_i in EdS with matching ICs must give
    # P_nu^{1/2}(a) = h0 a / a_i, i.e. R = 1 (up to the ln-a interpolation of
    # the stored spectra, O(dlna^2)).
    ai, a, h0 = 0.02, 0.1, 1.3
    c = eds(ai=ai)
    a_hist = ai * (a / ai) ** (np.arange(400) / 400)
    hist = (h0 * a_hist / ai)[:, None]
    r = O.nu_response([0.05], [h0 * a / ai], a, c, a_hist, hist, [[h0]], [[-ai ** -0.5]],
                      I_func=ONE)
    assert abs(r["R"][0] - 1.0) < 3e-6


def test_heavy_neutrinos_follow_cdm():
    # spec: delta_nu -> delta_cdm on large scales for heavy neutrinos.
    # With the exact I and m -> large, x -> 0 so I -> 1 and R -> 1 (EdS
    # growing mode as above).
    ai, a, h0 = 0.02, 0.1, 1.0
    c = eds(m=1e5, ai=ai)
    a_hist = ai * (a / ai) ** (np.arange(200) / 200)
    hist = (h0 * a_hist / ai)[:, None] * np.ones((1, 2))
    r = O.nu_response([0.01, 0.1], [h0 * a / ai] * 2, a, c, a_hist, hist,
                      [[h0, h0]], [[-ai ** -0.5] * 2])
    assert np.all(np.abs(r["R"] - 1.0) < 1e-5)


def _lcdm_inputs(nb=4, n_hist=10, ai=0.02, a=0.1, m=0.1):
    om = 0.3
    onu = 3 * m / (93.14 * 0.49)
    c = O.Cosmo(om - onu, onu, 0.7, (m, m, m), ai)
    kb = np.geomspace(0.01, 3.0, nb)
    a_hist = ai * (a / ai) ** (np.arange(n_hist) / n_hist)
    base = 10.0 / (1 + kb / 0.2) ** 1.5
    hist = (a_hist / ai)[:, None] * base[None, :]
    pi = np.tile(base / (1 + kb / 0.01) ** 2, (3, 1))
    ti = np.full((3, nb), -ai * math.sqrt(om / ai ** 3 + 1 - om))
    return c, kb, a_hist, hist, pi, ti, base * a / ai


def test_massless_limit():
    # spec: delta_nu -> 0 as M_nu -> 0.
    Rs = []
    for m in (0.1, 0.01, 1e-3):
        c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=3, m=m)
        Rs.append(O.nu_response(kb, cur, 0.1, c, ah, hist, pi, ti)["R"])
    Rs = np.array(Rs)
    assert np.all(np.diff(Rs, axis=0) < 0)
    assert np.all(Rs[-1] < 1e-3)
    c0 = O.Cosmo(0.3, 0.0, 0.7, (), 0.02)
    r0 = O.nu_response(kb, cur, 0.1, c0, ah, hist, pi, ti)
    assert np.all(r0["R"] == 0) and np.array_equal(r0["sqrtPM"], np.asarray(cur))


def _brute_J(kb, a, cosmo, m, a_nodes, h_nodes):
    """Independent route: J = 1.5 Om int_0^{sigma_max} I(kappa sigma) sigma
    P_M^{1/2}(a'(sigma)) a'(sigma) d sigma, sigma = s - s' (dtau' = a' ds'),
    on a fine geometric sigma grid, a'(sigma) from a dense monotone table,
    trapezoid rule."""
    om = cosmo.omega_m
    ai = cosmo.a_init
    la = np.linspace(math.log(ai), math.log(a), 400001)
    sig_tab = O.delta_s(np.exp(la), np.full_like(la, a), om)          # decreasing
    smax = sig_tab[0]
    sig = np.concatenate([[0.0], np.geomspace(smax * 1e-13, smax, 400000)])
    lna = np.interp(sig, sig_tab[::-1], la[::-1])
    ap = np.exp(lna)
    lnodes = np.log(np.asarray(a_nodes))
    out = []
    for b, k in enumerate(kb):
        h = np.interp(lna, lnodes, np.asarray(h_nodes)[:, b])        # const before node 0
        kappa = k * O.C_OVER_H0 * O.T_NU0_EV / m
        f = O.nu_I(kappa * sig) * sig * h * ap
        out.append(1.5 * om * integrate.trapezoid(f, sig))
    return np.array(out)


def test_integral_against_brute_force_quadrature():
    c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=4, n_hist=6)
    a = 0.1
    nodes = np.concatenate([ah, [a]])
    h = np.vstack([hist, cur[None, :]])
    J = O.response_integral(kb, a, c, 0.1, nodes, h)
    Jb = _brute_J(kb, a, c, 0.1, nodes, h)
    assert np.allclose(J, Jb, rtol=2e-7, atol=0)


def test_appendix_A_constant_potential():
    # App. A: in EdS with phi constant (P_M^{1/2} ~ a) and no initial neutrino
    # perturbation, the integral of Eq. P-final is delta_hdm = F delta_M with
    #   F = 6 / x_k^2 int_0^{x_max} x I(x) / (1 + x / x_k)^4 dx,
    #   x_k = 2 kappa / (a^2 H),  x_max = kappa (s - s_i) = x_k (sqrt(a/a_i) - 1)
    # (X_k = 2 k / (m a^2 H) times T_nu0).  This is exact for that history, so
    # the oracle's J / P_M^{1/2}(a) must reproduce it.  With x_max -> inf the
    # paper's fit 1 / (1 + k/k_fs)^2 agrees with F to < 12% and
    # F (k/k_fs)^2 -> 1 for k >> k_fs (Sec. 3.3.2).
    ai, a, m = 2.5e-5, 1e-2, 0.1
    c = eds(m=m, ai=ai)
    kfs = O.free_streaming_k(a, m, 1.0)
    ratios = np.array([0.3, 1.0, 3.0, 10.0, 100.0])
    kb = ratios * kfs
    la = np.linspace(math.log(ai), math.log(a), 1501)[:-1]
    hist = np.exp(la)[:, None] / a * np.ones((1, kb.size))
    nodes = np.concatenate([np.exp(la), [a]])
    h = np.vstack([hist, np.ones((1, kb.size))])
    J = O.response_integral(kb, a, c, m, nodes, h, epsrel=1e-10)
    kappa = kb * O.C_OVER_H0 * O.T_NU0_EV / m
    xk = 2 * kappa / (a * a * a ** -1.5)
    xmax = xk * (math.sqrt(a / ai) - 1)

    def F(xkk, upper):
        v, _ = integrate.quad(lambda x: x * O.nu_I(x) / (1 + x / xkk) ** 4, 0, upper,
                              epsabs=0, epsrel=1e-11, limit=400)
        return 6 / xkk ** 2 * v
    Ffin = np.array([F(q, u) for q, u in zip(xk, xmax)])
    Finf = np.array([F(q, np.inf) for q in xk])
    assert np.allclose(J, Ffin, rtol=3e-6, atol=0)
    assert np.all(np.abs(Finf * (1 + ratios) ** 2 - 1) < 0.12)
    assert abs(Finf[-1] * ratios[-1] ** 2 - 1) < 0.05


def test_second_iteration_small():
    # Sec. 4.3 (iii), App. B: the first iteration is converged to
    # O(f_nu (H dt)^2); check |P2 - P1| / P1 <= f_nu (H dt)^2 with H dt = dln a.
    c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=4, n_hist=20, a=0.1)
    a = 0.1
    prev_a = ah[-1]
    prev = O.nu_response(kb, cur * prev_a / a, prev_a, c, ah[:-1], hist[:-1], pi, ti)["sqrtPnu"]
    r1 = O.nu_response(kb, cur, a, c, ah, hist, pi, ti, sqrtPnu_prev=prev, iters=1)
    r2 = O.nu_response(kb, cur, a, c, ah, hist, pi, ti, sqrtPnu_prev=prev, iters=2)
    Hdt = math.log(a / prev_a)
    rel = np.abs(r2["sqrtPnu"] - r1["sqrtPnu"]) / np.abs(r1["sqrtPnu"])
    assert np.all(rel <= c.f_nu * Hdt ** 2)
    assert np.all(rel > 0)


def test_species_weighting():
    # Sec. 6.2: several species are summed with weights Omega_nu,i / Omega_nu.
    c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=3)
    one = O.Cosmo(c.omega_cdm, c.omega_nu, c.h, (0.3,), c.a_init)
    r3 = O.nu_response(kb, cur, 0.1, O.Cosmo(c.omega_cdm, c.omega_nu, c.h, (0.1, 0.1, 0.1),
                                              c.a_init), ah, hist, pi, ti)
    # degenerate species of mass m equal one species of mass m
    r1 = O.nu_response(kb, cur, 0.1, O.Cosmo(c.omega_cdm, c.omega_nu, c.h, (0.1,), c.a_init),
                       ah, hist, pi[:1], ti[:1])
    assert np.allclose(r3["R"], r1["R"], rtol=1e-12)
    assert one.species_weights().tolist() == [1.0]


def test_empty_bins_and_ic_only():
    c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=3)
    cur = np.array(cur)
    cur[1] = 0.0
    r = O.nu_response(kb, cur, 0.1, c, ah, hist, pi, ti)
    assert r["R"][1] == 0.0
    # no history, a = a_i: P_nu = P_nu,i exactly (I(0) = 1, s - s_i = 0)
    r0 = O.nu_response(kb, cur, c.a_init, c, [], np.zeros((0, 3)), pi, ti)
    assert np.allclose(r0["sqrtPnu"], pi[0], rtol=1e-14)
    with pytest.raises(ValueError):
        O.nu_response(kb, cur, 0.05, c, ah, hist, pi, ti)      # a < last history node


def test_species_weights_follow_the_mass():
    # Sec. 2.1: Omega_nu h^2 = sum m / 93.14 eV, so species i carries the
    # fraction m_i / M_nu of the neutrino density.  A light second species
    # (m_2 = m_1 / 50: free streaming suppresses its response by ~(m_2/m_1)^2)
    # must leave the heavy species' response scaled by m_1 / M_nu ~ 0.98 plus
    # at most a percent of m_2 / M_nu; equal weights (1 / n_species) would
    # halve it.
    c, _, ah, hist, _, ti, _ = _lcdm_inputs(nb=4)
    kb = np.array([0.01, 0.02, 0.04, 0.08])
    cur = 10.0 / (1 + kb / 0.2) ** 1.5 * 0.1 / c.a_init
    pi = np.tile(10.0 / (1 + kb / 0.2) ** 1.5 / (1 + kb / 0.01) ** 2, (3, 1))
    m1, m2 = 0.1, 0.002
    one = O.Cosmo(c.omega_cdm, c.omega_nu, c.h, (m1,), c.a_init)
    r1 = O.nu_response(kb, cur, 0.1, one, ah, hist, pi[:1], ti[:1])
    w1, w2 = m1 / (m1 + m2), m2 / (m1 + m2)
    for masses in ((m1, m2), (m2, m1)):      # the weight goes with its own species
        two = O.Cosmo(c.omega_cdm, c.omega_nu, c.h, masses, c.a_init)
        assert np.allclose(two.species_weights(), np.array(masses) / (m1 + m2), rtol=1e-15)
        # same initial arrays for both species: the first-iteration guess is unchanged
        r2 = O.nu_response(kb, cur, 0.1, two, ah, hist, pi[:2], ti[:2])
        extra = r2["R"] / r1["R"] - w1
        assert np.all(extra >= 0) and np.all(extra < 0.01 * w2)


def test_hierarchy_is_the_mass_weighted_sum_of_species():
    # Sec. 6.2 / Table 1 (S03NH masses): a hierarchy of unequal masses sums
    # the single-species responses with weights m_i / M_nu.  The single-species
    # runs use the same first-iteration guess (identical initial arrays).
    c, kb, ah, hist, pi, ti, cur = _lcdm_inputs(nb=3)
    masses = (0.022, 0.024, 0.054)
    tot = sum(masses)
    full = O.nu_response(kb, cur, 0.1, O.Cosmo(c.omega_cdm, c.omega_nu, c.h, masses, c.a_init),
                         ah, hist, pi, ti)
    parts = [O.nu_response(kb, cur, 0.1, O.Cosmo(c.omega_cdm, c.omega_nu, c.h, (m,), c.a_init),
                           ah, hist, pi[:1], ti[:1])["sqrtPnu"] for m in masses]
    want = sum(m / tot * p for m, p in zip(masses, parts))
    assert np.allclose(full["sqrtPnu"], want, rtol=1e-9)
    # the heaviest species responds most: R ordered by mass in every bin
    Rs = [p / cur for p in parts]
    assert np.all(Rs[0] < Rs[1]) and np.all(Rs[1] < Rs[2])
