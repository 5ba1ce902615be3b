"""GPU tests of the learned response surrogate through the C ABI: the network's
forward pass, gradient and Adam step against the FP64 oracle (same BF16
weights), the features against the oracle's definition, pm_set_power with the
exact response against the oracle, and a short training run that shows what
the surrogate gains over the exact integral and what it costs in accuracy."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib  # noqa: E402
from oracle import mlp_oracle as MO  # noqa: E402
from oracle import pm_oracle as O  # noqa: E402
from paper_1209_0461_gb300 import nupm, surrogate, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


def _random_net(seed, n=1000):
    rng = np.random.default_rng(seed)
    theta = surrogate.init_params(seed)
    theta[128 * 12:128 * 12 + 128] = rng.normal(scale=0.1, size=128)          # b1
    theta[-1] = 0.3                                                              # b3
    X = rng.normal(size=(n, 12)) * np.linspace(0.5, 3, 12) + np.linspace(-1, 1, 12)
    y = rng.normal(size=n)
    mu = np.linspace(-1, 1, 12).astype(np.float32)
    sig = np.linspace(0.5, 3, 12).astype(np.float32)
    return theta, X.astype(np.float32), y.astype(np.float32), (mu, sig, np.float32(0.2), np.float32(1.7))


def _norm64(norm):
    mu, sig, ym, ys = norm
    return (mu.astype(np.float64), sig.astype(np.float64), float(ym), float(ys))


@pytest.mark.parametrize("n", [1, 31, 1000])
def test_forward_matches_oracle(n):
    theta, X, _, norm = _random_net(1, n)
    m = nupm.MLP()
    m.set_params(theta)
    m.set_norm(*norm)
    got = m.forward(torch.from_numpy(X).cuda()).double().cpu().numpy()
    ref = MO.predict_lnR(theta.astype(np.float64), (norm[0].astype(np.float64), norm[1].astype(np.float64),
                                                     float(norm[2]), float(norm[3])), X)
    assert np.max(np.abs(got - ref)) < 2e-5 * (1 + np.max(np.abs(ref))), np.max(np.abs(got - ref))
    m.close()


def test_gradient_matches_oracle():
    theta, X, y, norm = _random_net(2, 777)
    m = nupm.MLP()
    m.set_params(theta)
    m.set_norm(*norm)
    g, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    g = g.double().cpu().numpy()
    mu, sig, ym, ys = _norm64(norm)
    P = MO.effective(theta.astype(np.float64), 12, 128)
    Xh = (X.astype(np.float64) - mu) / sig
    L, gr = MO.loss_and_grad(P, Xh, (y.astype(np.float64) - ym) / ys)
    gref = MO.pack(gr, 12, 128)
    assert abs(float(loss.item()) - L) < 1e-5 * L
    assert np.linalg.norm(g - gref) < 1e-4 * np.linalg.norm(gref)
    # every parameter group, relative to its own scale
    o = 0
    for name, shape in MO.param_sizes(12, 128):
        k = int(np.prod(shape))
        assert np.linalg.norm(g[o:o + k] - gref[o:o + k]) <= 1e-4 * np.linalg.norm(gref[o:o + k]) + 1e-9, name
        o += k
    # deterministic: a second evaluation is bit-identical
    g2, _ = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    assert np.array_equal(g2.double().cpu().numpy(), g)
    m.close()


def test_adam_step_matches_oracle():
    theta, X, y, norm = _random_net(3, 512)
    m = nupm.MLP()
    m.set_params(theta)
    m.set_norm(*norm)
    g, _ = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    g = g.double().cpu().numpy()
    lr = 1e-3
    m.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), lr)
    t1 = m.get_params().astype(np.float64)
    ref, _, _ = MO.adam_step(theta.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    big = np.abs(g) > 1e-5
    assert np.max(np.abs(t1 - ref)[big]) < 1e-6
    assert np.max(np.abs(t1 - theta)) <= lr * 1.001
    m.close()


def _power_ctx(w, kb, n_hist_max=32):
    pi, ti = synth.nu_initial_at(kb, w)
    return nupm.PM(32, 8, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species, a_init=w.a_init,
                   n_kbins=kb.size, n_hist_max=n_hist_max, precision="fp64", sqrtPnu_init=pi,
                   theta_over_delta_init=ti), pi, ti


def test_set_power_response_and_features_match_oracle():
    w, kb, scen = synth.surrogate_group(5, 3, n_kbins=48, n_hist_max=32)
    pm, pi, ti = _power_ctx(w, kb)
    unit = 32.0 ** 6 / w.box ** 3
    cos = O.Cosmo(w.omega_cdm, w.omega_nu, w.h, w.masses, w.a_init)
    for s in scen:
        pm.set_power(np.ones(kb.size), kb, s["sqrtPcdm"] ** 2 * unit)
        hist = torch.from_numpy(np.ascontiguousarray(s["hist"])).cuda()
        R = torch.empty(kb.size, dtype=torch.float64, device="cuda")
        pm.nu_response(s["a"], s["a_hist"], hist, ratio=R)
        ref = O.nu_response(kb, s["sqrtPcdm"], s["a"], cos, s["a_hist"], s["hist"], pi, ti)
        # Gauss-Legendre panels against adaptive quadrature, down to R ~ 1e-6 at k = 20 h/Mpc
        assert np.allclose(R.cpu().numpy(), ref["R"], rtol=1e-7, atol=0)
        X = pm.response_features(s["a"], s["a_hist"], hist).double().cpu().numpy()
        Xr = MO.features(kb, s["a"], w.m_nu_total, w.omega_nu, w.a_init, s["a_hist"], s["hist"], s["sqrtPcdm"])
        assert np.allclose(X, Xr, rtol=2e-7, atol=2e-6), np.max(np.abs(X - Xr))
    # a kick needs a real deposit after pm_set_power
    with pytest.raises(nupm.PMError) as e:
        pos = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
        pm.kick(pos, torch.zeros_like(pos), scen[-1]["a"], 0.01)
    assert e.value.code == -7
    pm.close()


def test_deposit_restores_lattice_bins_after_set_power():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], n_hist=4)
    parts = synth.particles(w)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, precision="fp64",
                 sqrtPnu_init=synth.nu_initial(w)[0], theta_over_delta_init=synth.nu_initial(w)[1])
    pos = torch.from_numpy(parts["pos64"]).cuda()
    pm.deposit(pos)
    b0 = pm.bins()
    pm.set_power(np.full(w.n_kbins, 3.0), np.full(w.n_kbins, 0.3), np.ones(w.n_kbins))
    assert np.all(pm.bins()[0] == 3.0)
    pm.deposit(pos)
    b1 = pm.bins()
    assert all(np.array_equal(x, y) for x, y in zip(b0, b1))
    pm.close()


def test_surrogate_trains_and_stands_in_for_the_integral():
    # a reduced training set (the bench trains on 1e6 samples)
    X, y, ids, fnu = surrogate.build_set(48, 32, seed0=100, n_kbins=128, n_hist_max=128)
    Xv, yv, _, fv = surrogate.build_set(4, 8, seed0=900, n_kbins=128, n_hist_max=128)
    m = nupm.MLP()
    m.set_params(surrogate.init_params(0))
    surrogate.fit_norm(m, X, y)
    hist = surrogate.train(m, X, y, epochs=60, batch=2048, lr0=3e-3)
    assert hist[-1] < 0.05 * hist[0]
    rel, force = surrogate.errors(m, Xv, yv, fv)
    print(f"held-out: median |dR|/R {np.median(rel):.3e}, p99 {np.percentile(rel, 99):.3e}, "
          f"max f|dR|/(1-f+fR) {np.max(force):.3e}")
    assert np.median(rel) < 0.05
    assert np.percentile(force, 99) < 5e-3
    # pm_nu_response_mlp = features -> network -> exp, and it prepares a kick
    w, kb, scen = synth.surrogate_group(901, 1, n_kbins=128, n_hist_max=128)
    pm, _, _ = _power_ctx(w, kb, 128)
    s = scen[0]
    unit = 32.0 ** 6 / w.box ** 3
    pm.set_power(np.ones(kb.size), kb, s["sqrtPcdm"] ** 2 * unit)
    h = torch.from_numpy(np.ascontiguousarray(s["hist"])).cuda()
    Rm = torch.empty(kb.size, dtype=torch.float64, device="cuda")
    pm.nu_response_mlp(m, s["a"], s["a_hist"], h, ratio=Rm)
    Xf = pm.response_features(s["a"], s["a_hist"], h)
    lnR = m.forward(Xf).double().cpu().numpy()
    assert np.allclose(Rm.cpu().numpy(), np.exp(lnR), rtol=1e-6)
    # gain: the surrogate's cost does not grow with the history, the integral's does
    a_hist = w.a_init * (s["a"] / w.a_init) ** (np.arange(128) / 128)
    hist128 = torch.from_numpy(np.ascontiguousarray(
        np.interp(np.log(a_hist), np.log(s["a_hist"]), s["hist"][:, 0])[:, None] * np.ones(kb.size))).cuda()

    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t_exact = timed(lambda: pm.nu_response(s["a"], a_hist, hist128))
    t_mlp = timed(lambda: pm.nu_response_mlp(m, s["a"], a_hist, hist128))
    print(f"response at 128 history nodes: exact {t_exact * 1e3:.3f} ms, surrogate {t_mlp * 1e3:.3f} ms")
    assert t_mlp < t_exact
    pm.close()
    m.close()
