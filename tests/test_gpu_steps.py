"""The step loop either side of the kick (Sec. 4.3: evolve, steps (ii)-(iv),
store P_M, repeat) and the Sec. 4.4 background, through the C ABI against the
oracle:

  * pm_drift bit for bit against the oracle's drift (FP64 and int cell +
    FP32 offset), face crossings and the offset-rounds-to-one case included;
  * pm_step runs of several leapfrog steps from a stored history against the
    oracle's pm_step loop: history rows, velocities and positions;
  * a single small mode grown by pm_step on the GPU follows D(a) to 1%;
  * PM_RELATIVISTIC (Eq. relativistic energy density and radiation in H(a))
    against the oracle's background: kick/drift factors, response, forces."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib, cosmo_of, force_errors, gpu_kick, make_inputs, oracle_kick  # noqa: E402
from oracle import pm_oracle as O  # noqa: E402
from paper_1209_0461_gb300 import nupm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


def _ctx(w, flags=0, n_hist_max=64, npart=None):
    pi, ti = synth.nu_initial(w)
    return nupm.PM(w.ngrid, npart or w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                   m_nu=w.m_species or None, a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=n_hist_max,
                   precision=w.precision, flags=flags, sqrtPnu_init=pi, theta_over_delta_init=ti)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_drift_bit_exact(prec):
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"drift_{prec}", precision=prec)
    parts = synth.particles(w)
    rng = np.random.default_rng(11)
    vel = parts["vel"] * 40.0 + rng.normal(0, 50.0, parts["vel"].shape)   # many cell and face crossings
    ds = 0.73
    pm = _ctx(w)
    if prec == "fp64":
        pos = parts["pos64"].copy()
        pos[0, :4] = [0.0, 1e-13, w.box - 1e-13, np.nextafter(w.box, 0)]   # face cases
        vel[0, :4] = [-1e-15, -1e-13, 1e-13, 1e-300]
        pt = torch.from_numpy(pos).to(DEV)
        vt = torch.from_numpy(vel).to(DEV)
        pm.drift(pt, vt, ds)
        pm.check()
        want = O.drift_f64(pos, vel, ds, w.box)
        got = pt.cpu().numpy()
        assert np.array_equal(got, want)
        assert np.all((got >= 0) & (got < w.box))
    else:
        packed = synth.to_cell_offset(parts["pos64"], w.box, w.ngrid)
        cell, off = synth.split_cell_offset(packed)
        off[0, :3] = [0.0, np.float32(0.5), np.nextafter(np.float32(1), np.float32(0))]
        packed[3:] = off.view(np.int32)
        v32 = vel.astype(np.float32)
        g = np.float32(ds / (w.box / w.ngrid))
        v32[0, :3] = [-2.0 ** -30 / g, 0.25 / g, 1e-7 / g]
        pt = torch.from_numpy(packed).to(DEV)
        vt = torch.from_numpy(v32).to(DEV)
        pm.drift(pt, vt, ds)
        pm.check()
        cw, ow = O.drift_cell(cell, off, v32, g, w.ngrid)
        got = pt.cpu().numpy()
        gc, go = synth.split_cell_offset(got)
        assert np.array_equal(gc, cw)
        assert np.array_equal(go.view(np.int32), ow.view(np.int32))
        assert gc[0, 0] == cell[0, 0] and go[0, 0] == 0.0        # o' rounds to 1: offset 0, same cell
    pm.close()


def test_drift_rejects_bad_offsets_without_moving():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="drift_bad", precision="fp32")
    parts = synth.particles(w)
    packed = synth.to_cell_offset(parts["pos64"], w.box, w.ngrid)
    packed[3, 7] = np.float32(1.5).view(np.int32)
    before = packed.copy()
    pm = _ctx(w)
    pt = torch.from_numpy(packed).to(DEV)
    vt = torch.ones((3, w.npart), dtype=torch.float32, device=DEV)
    pm.drift(pt, vt, 0.1)
    with pytest.raises(nupm.PMError) as e:
        pm.check()
    assert e.value.code == -2
    got = pt.cpu().numpy()
    assert np.array_equal(got[:, 7], before[:, 7])
    assert not np.array_equal(got[:, 8], before[:, 8])
    pm.close()


def _run_steps(w, n_steps, a1, prec_tol, rel=False):
    """pm_step on the GPU and the oracle's pm_step loop from the same stored
    history (up to a_kick) over n_steps leapfrog steps to a1."""
    flags = nupm.PM_RELATIVISTIC if rel else 0
    inp = make_inputs(w)
    a0 = w.a_kick
    a_steps = np.exp(np.linspace(math.log(a0), math.log(a1), n_steps + 1))
    cos = O.Cosmo(w.omega_cdm, w.omega_nu, w.h, w.masses, w.a_init, relativistic=rel)
    kicks, drifts = O.leapfrog_factors(a_steps, cos)
    pm = _ctx(w, flags=flags, n_hist_max=w.n_hist + n_steps + 1)
    # the library's own factors agree with the oracle's
    mid = [math.sqrt(a_steps[j] * a_steps[j + 1]) for j in range(n_steps)]
    lo, hi = [a_steps[0]] + mid, mid + [a_steps[-1]]
    kg = [pm.kick_factor(l, h) for l, h in zip(lo, hi)]
    dg = [pm.drift_factor(a_steps[j], a_steps[j + 1]) for j in range(n_steps)] + [0.0]
    assert np.allclose(kg, kicks, rtol=1e-12, atol=0) and np.allclose(dg, drifts, rtol=1e-12, atol=0)
    fp64 = w.precision == "fp64"
    if fp64:
        pos = torch.from_numpy(inp["pos64"]).to(DEV)
        vel = torch.from_numpy(inp["vel"]).to(DEV)
        run = O.StepRun("fp64", inp["pos64"].copy(), inp["vel"].copy(), list(inp["a_hist"]), list(inp["hist"]))
    else:
        packed = synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)
        pos = torch.from_numpy(packed).to(DEV)
        v32 = inp["vel"].astype(np.float32)
        vel = torch.from_numpy(v32).to(DEV)
        run = O.StepRun("fp32", synth.split_cell_offset(packed), v32.astype(np.float64), list(inp["a_hist"]),
                        list(inp["hist"]))
    pm.history_set(inp["a_hist"], torch.from_numpy(np.ascontiguousarray(inp["hist"])).to(DEV))
    for a, K, S in zip(a_steps, kg, dg):
        pm.step(pos, vel, a, K, S)
        O.pm_step(run, w.ngrid, w.box, a, K, S, cos, w.n_kbins, inp["pi"], inp["ti"])
    pm.check()
    ah, rows, prev = pm.history_get()
    assert np.array_equal(ah, np.array(run.a_hist))
    got_rows = rows.cpu().numpy()
    want_rows = np.array(run.hist)
    nz = want_rows != 0
    assert np.array_equal(got_rows != 0, nz)
    rel_rows = np.abs(got_rows[nz] / want_rows[nz] - 1)
    vg = vel.cpu().numpy().astype(np.float64)
    dv = np.sqrt(((vg - run.vel) ** 2).sum(0))
    verr = float(np.sqrt((dv ** 2).mean()) / np.sqrt((run.vel ** 2).sum(0).mean()))
    if fp64:
        xg = pos.cpu().numpy()
        dx = np.abs(xg - run.pos)
        dx = np.minimum(dx, w.box - dx)
    else:
        gc, go = synth.split_cell_offset(pos.cpu().numpy())
        xg = gc + go.astype(np.float64)
        xo = run.pos[0] + run.pos[1].astype(np.float64)
        dx = np.abs(xg - xo)
        dx = np.minimum(dx, w.ngrid - dx) * (w.box / w.ngrid)
    print(f"{w.name} rel={rel}: rows max rel {rel_rows.max():.2e}, vel rms rel {verr:.2e}, "
          f"pos max {dx.max():.2e} Mpc/h")
    assert rel_rows.max() < prec_tol
    assert verr < prec_tol
    assert dx.max() < prec_tol * w.box
    pm.close()
    return run


def test_step_loop_fp64_against_oracle():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="steps64", n_hist=8, a_kick=0.05)
    _run_steps(w, 6, 0.1, 1e-8)


def test_step_loop_fp32_hierarchy_against_oracle():
    w = synth.hierarchy(synth.with_(synth.WORKLOADS["pm32_fp64"], name="steps32", ngrid=64, npart_side=64,
                                    box=128.0, precision="fp32", n_hist=8, n_kbins=24, a_kick=0.05))
    _run_steps(w, 5, 0.1, 2e-4)


def test_step_loop_relativistic_background():
    w = synth.hierarchy(synth.with_(synth.WORKLOADS["pm32_fp64"], name="steps_rel", n_hist=6, a_kick=0.04,
                                    n_kbins=16))
    _run_steps(w, 3, 0.06, 1e-8, rel=True)


def test_history_full_and_order_errors():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="hist_err", n_hist=4)
    inp = make_inputs(w)
    pm = _ctx(w, n_hist_max=5)
    pos = torch.from_numpy(inp["pos64"]).to(DEV)
    vel = torch.from_numpy(inp["vel"]).to(DEV)
    pm.history_set(inp["a_hist"], torch.from_numpy(np.ascontiguousarray(inp["hist"])).to(DEV))
    with pytest.raises(nupm.PMError) as e:
        pm.step(pos, vel, float(inp["a_hist"][-1]), 0.0, 0.0)      # not after the last stored a
    assert e.value.code == -2
    pm.step(pos, vel, w.a_kick, 0.0, 0.0)
    with pytest.raises(nupm.PMError) as e:
        pm.step(pos, vel, w.a_kick * 1.1, 0.0, 0.0)                # history full
    assert e.value.code == -2
    pm.close()


def test_single_mode_growth_through_the_gpu_step_loop():
    # the oracle's pin (tests/test_oracle_steps.py) run by pm_step: CDM only,
    # a 1% sine mode at a_i = 0.02 grown to a = 0.1 in 40 leapfrog steps
    n, L, om, ai, af, nsteps = 32, 256.0, 0.3, 0.02, 0.1, 40
    k0 = 2 * math.pi / L
    amp = 0.01 / k0
    q1 = (np.arange(n) + 0.5) * L / n
    qz, qy, qx = np.meshgrid(q1, q1, q1, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()])
    psi = np.zeros_like(q)
    psi[0] = amp * np.sin(k0 * q[0])
    Di, fi = synth.growth(ai, om)
    Df, _ = synth.growth(af, om)
    H = math.sqrt(om / ai ** 3 + 1 - om)
    pm = nupm.PM(n, n ** 3, L, om, 0.0, 0.7, 0.0, 0, a_init=ai, n_kbins=8, n_hist_max=nsteps + 1)
    pos = torch.from_numpy(np.mod(q + psi, L)).to(DEV)
    vel = torch.from_numpy(ai * ai * H * fi * psi).to(DEV)
    a_steps = np.exp(np.linspace(math.log(ai), math.log(af), nsteps + 1))
    mid = [math.sqrt(a_steps[j] * a_steps[j + 1]) for j in range(nsteps)]
    lo, hi = [a_steps[0]] + mid, mid + [a_steps[-1]]
    for j, a in enumerate(a_steps):
        S = pm.drift_factor(a, a_steps[j + 1]) if j < nsteps else 0.0
        pm.step(pos, vel, a, pm.kick_factor(lo[j], hi[j]), S)
    pm.check()
    x = pos.cpu().numpy()
    disp = (x[0] - q[0] + L / 2) % L - L / 2
    growth = (disp * np.sin(k0 * q[0])).sum() / (np.sin(k0 * q[0]) ** 2).sum() / amp
    print(f"growth {growth:.5f} vs D ratio {Df / Di:.5f}")
    assert abs(growth / (Df / Di) - 1) < 0.01
    pm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_relativistic_background_kick(prec):
    # Sec. 4.4 background with the S03NH hierarchy: response per bin and forces
    # against the oracle with the same background; the background changes R
    w = synth.hierarchy(synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"rel_{prec}", precision=prec, n_hist=6,
                                    n_kbins=16, ngrid=32 if prec == "fp64" else 64,
                                    npart_side=32 if prec == "fp64" else 64))
    inp = make_inputs(w)
    g = gpu_kick(w, inp, flags=0x4 | nupm.PM_RELATIVISTIC)
    cos = O.Cosmo(w.omega_cdm, w.omega_nu, w.h, w.masses, w.a_init, relativistic=True)
    if prec == "fp64":
        c, q = O.quantise_positions_f64(inp["pos64"], w.box, w.ngrid)
        vel = inp["vel"]
    else:
        cell, off = synth.split_cell_offset(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid))
        c, q = O.quantise_positions_cell(cell, off, w.ngrid)
        vel = inp["vel"].astype(np.float32).astype(np.float64)
    r = O.pm_kick(c, q, vel, w.ngrid, w.box, w.a_kick, 0.01, cos, w.n_kbins, inp["a_hist"], inp["hist"],
                  inp["pi"], inp["ti"])
    ne = r.bins["nonempty"]
    relR = np.abs(g["R"][ne] / r.response["R"][ne] - 1)
    emax, erms = force_errors(g["acc"], r.acc)
    r_nr = oracle_kick(w, inp)
    shift = np.abs(r_nr.response["R"][ne] / r.response["R"][ne] - 1).max()
    print(f"{prec}: R max rel {relR.max():.2e} (background shifts R by {shift:.2e}), force max {emax:.2e}")
    assert relR.max() < (1e-9 if prec == "fp64" else 1e-5)
    assert (emax if prec == "fp64" else erms) < (1e-5 if prec == "fp64" else 2e-4)
    assert shift > 1e-4
