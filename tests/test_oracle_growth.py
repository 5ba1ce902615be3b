"""Multi-step pin of the oracle kick: a single small-amplitude mode in a
CDM-only run grows with the linear growth factor D(a) (north star: "linear
growth of a single seeded mode in a CDM-only run").  The drift used here is a
test-only helper, not part of the kick."""
import math

import numpy as np
from scipy import integrate

from oracle import pm_oracle as O


def lcdm_growth(a, om):
    H = lambda t: math.sqrt(om / t ** 3 + 1 - om)
    I = lambda x: integrate.quad(lambda t: 1.0 / (t * H(t)) ** 3, 0, x, epsrel=1e-12)[0]
    Ia = I(a)
    D = H(a) * Ia
    f = -1.5 * om / (a ** 3 * H(a) ** 2) + 1.0 / (a * a * H(a) ** 3 * Ia)
    return D, f


def test_single_mode_linear_growth():
    n, L, om = 32, 256.0, 0.3
    cos = O.Cosmo(om, 0.0, 0.7, (), 0.02)
    ai, af, nsteps = 0.02, 0.1, 40
    k0 = 2 * math.pi / L
    amp = 0.01 / k0                      # delta = -D psi' ~ 1% at a_i
    q1 = (np.arange(n) + 0.5) * L / n
    qz, qy, qx = np.meshgrid(q1, q1, q1, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()])
    psi = np.zeros_like(q)
    psi[0] = amp * np.sin(k0 * q[0])
    Di, fi = lcdm_growth(ai, om)
    Df, _ = lcdm_growth(af, om)
    H = lambda a: math.sqrt(om / a ** 3 + 1 - om)
    x = q + psi
    u = ai * ai * H(ai) * fi * psi            # u = a^2 dx/dt for x = q + (D/Di) psi
    lna = np.linspace(math.log(ai), math.log(af), nsteps + 1)
    a_steps = np.exp(lna)

    def acc(xx, a):
        c, w = O.quantise_positions_f64(xx, L, n)
        F = O.cic_deposit(c, w, n)
        spec = O.forward_fft(O.density_contrast(F, xx.shape[1]))
        nk = 8
        accs = O.green_gradient(spec, L, a, cos, np.ones(nk), np.zeros(nk), np.zeros(nk, bool))
        return np.stack([O.cic_interpolate(O.inverse_fft(g, n), c, w) for g in accs])

    g = acc(x, ai)
    for a0, a1 in zip(a_steps[:-1], a_steps[1:]):
        am = math.sqrt(a0 * a1)
        u = u + g * O.kick_factor(a0, am, om)
        x = x + u * O.drift_factor(a0, a1, om)
        g = acc(x, a1)
        u = u + g * O.kick_factor(am, a1, om)
    disp = x[0] - q[0]
    disp = (disp + L / 2) % L - L / 2
    fit = (disp * np.sin(k0 * q[0])).sum() / (np.sin(k0 * q[0]) ** 2).sum()
    growth = fit / amp
    assert abs(growth / (Df / Di) - 1) < 0.01
    # transverse components stay zero
    assert np.max(np.abs(x[1] - q[1])) < 1e-9 and np.max(np.abs(x[2] - q[2])) < 1e-9
