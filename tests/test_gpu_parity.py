"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Tolerances: deposit bit-exact; FP64 forces and response
max-relative 1e-5; FP32 forces RMS-relative 2e-4 (as the kick's accuracy
contract states)."""
import math

import numpy as np
import pytest

from oracle import pm_oracle as O
from paper_1209_0461_gb300 import nupm, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from gpu_common import (KEEP_DEPOSIT, FUSED_GATHER, SPECTRAL_GRADIENT, UNFUSED_DEPOSIT, build_lib,  # noqa: E402
                        cosmo_of, force_errors, gpu_kick, make_inputs, oracle_kick)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


def _check_common(w, g, r, fp64):
    # a1: bit-exact fixed-point deposit, exact mass conservation
    assert np.array_equal(g["F"].astype(np.int64), r.F)
    assert int(g["F"].astype(object).sum()) == g["acc"].shape[1] * 2 ** 48
    # bins: identical thresholds and mode counts
    assert np.array_equal(g["T"], r.bins["T"])
    cnt, ks, ps = g["bins"]
    assert np.array_equal(cnt, r.bins["count"])
    # FP64 sums of up to ~1e5 |k| values per bin in different orders
    assert np.allclose(ks, r.bins["ksum"], rtol=1e-12, atol=0)
    tol_p = 1e-10 if fp64 else 2e-5
    assert np.allclose(ps, r.bins["psum"], rtol=tol_p, atol=1e-300)
    # spectrum
    spec_ref = r.extras["spec"]
    d = np.abs(g["spec"] - spec_ref)
    scale = np.sqrt(np.mean(np.abs(spec_ref) ** 2))
    if fp64:
        assert d.max() < 1e-11 * scale
    else:
        assert np.sqrt(np.mean(d ** 2)) < 2e-6 * scale
    # a4: response per bin
    ne = r.bins["nonempty"]
    for key, gk in (("R", "R"), ("sqrtPnu", "Pnu"), ("sqrtPM", "PM")):
        ref = r.response[key]
        got = g[gk]
        rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        assert np.all(rel[ne] < (1e-9 if fp64 else 1e-5)), (key, rel[ne].max())
        assert np.all(got[~ne] == 0)
    # a5-a7: forces and the kick
    emax, erms = force_errors(g["acc"], r.acc)
    if fp64:
        assert emax < 1e-5, emax
    else:
        assert erms < 2e-4, erms
    dv = g["vel"] - g["vel0"]
    scale_v = np.max(np.abs(dv)) + 1e-300
    assert np.max(np.abs(dv - g["acc"] * 0.01)) < (1e-12 if fp64 else 1e-5) * scale_v


def test_plain_fp64_kick_32():
    w = synth.WORKLOADS["pm32_fp64"]
    inp = make_inputs(w)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    _check_common(w, g, r, True)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_kick_192_mixed_radix(prec):
    # 192^3 grid (radix-3 transforms, non-power-of-two wraps) against the oracle,
    # a ragged particle count and the batched form's box range
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"pm192_{prec}", ngrid=192, npart_side=96,
                    box=350.0, precision=prec, n_hist=8, n_kbins=48, m_nu_total=0.15)
    inp = make_inputs(w, npart=96 ** 3 - 5)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    _check_common(w, g, r, prec == "fp64")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_clustered_kick_contention(prec):
    # Zel'dovich at a = 1 in a 64 Mpc/h box: 57% of the cells empty, up to ~35
    # particles in one cell -- the shared-memory tile sums see heavy contention
    # and carries; the deposit must stay bit-exact
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"cl64_{prec}", ngrid=64, npart_side=64,
                    box=64.0, precision=prec, n_hist=8, n_kbins=24, clustered=True)
    inp = make_inputs(w)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    _check_common(w, g, r, prec == "fp64")


def test_fp32_kick_ragged_64():
    # 64^3 grid, FP32 form, a particle count that is not a multiple of any block size
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="pm64_fp32", ngrid=64, npart_side=64,
                    box=128.0, precision="fp32", n_hist=8, n_kbins=24)
    inp = make_inputs(w, npart=64 ** 3 - 37)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    _check_common(w, g, r, False)


@pytest.mark.parametrize("prec,n", [(p, n) for p in ("fp64", "fp32") for n in (16, 32, 64, 128, 192, 256)] +
                         [("fp32", 512)])
def test_fft_and_bins_sizes(n, prec):
    # spectrum of the deposit and its bin sums at every built grid size, both
    # precisions (the FP32 sums of 128^3 .. 1024^3 grids stage rows by TMA)
    w = synth.Workload(f"fft{n}", n, min(n, 64), 2.0 * n, 0.15, 3, 2, 12, prec)
    inp = make_inputs(w)
    g = gpu_kick(w, inp)
    F = g["F"].astype(np.int64)
    spec = O.forward_fft(O.density_contrast(F, inp["pos64"].shape[1]))
    d = np.abs(g["spec"] - spec)
    scale = np.sqrt(np.mean(np.abs(spec) ** 2))
    if prec == "fp64":
        assert d.max() < 1e-11 * scale
    else:
        assert np.sqrt(np.mean(d ** 2)) < 2e-6 * scale
    b = O.bin_power(spec, w.box, w.n_kbins)
    cnt, ks, ps = g["bins"]
    assert np.array_equal(cnt, b["count"])
    ne = b["count"] > 0
    rk = np.max(np.abs(ks[ne] - b["ksum"][ne]) / b["ksum"][ne])
    rp = np.max(np.abs(ps[ne] - b["psum"][ne]) / b["psum"][ne])
    print(f"{prec} N={n}: ksum max rel {rk:.1e}, psum max rel {rp:.1e}")
    # FP64 sums of up to ~7e7 |k| values per bin, summed in different orders
    # (the oracle's bincount runs sequentially: error up to ~n eps)
    assert rk < 1e-10
    assert rp < (1e-10 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("flags", [KEEP_DEPOSIT, KEEP_DEPOSIT | SPECTRAL_GRADIENT])
def test_inverse_fields_against_oracle(flags):
    # force grids: by default the 4-point stencil on the potential grid, with
    # PM_SPECTRAL_GRADIENT the inverse transforms of -i D(k) phi(k)
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], n_hist=6)
    inp = make_inputs(w)
    g = gpu_kick(w, inp, keep_fields=True, n_hist=6, flags=flags)
    r = oracle_kick(w, inp, n_hist=6)
    for c in range(3):
        ref = r.extras["fields"][c]
        assert np.max(np.abs(g["fields"][c] - ref)) < 1e-11 * np.max(np.abs(ref))
    if flags & SPECTRAL_GRADIENT:
        assert "phi" not in g
        return
    # the potential grid itself: inverse transform of G delta_M (Eq. Poisson)
    phi_k = O.potential_spectrum(r.extras["spec"], w.box, w.a_kick, cosmo_of(w), r.bins["k"], r.response["R"],
                                 r.bins["nonempty"])
    ref = O.inverse_fft(phi_k, w.ngrid)
    assert np.max(np.abs(g["phi"] - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,n", [("fp64", 64), ("fp32", 128), ("fp32", 192)])
def test_real_space_gradient_equals_spectral(prec, n):
    # the gather's stencil on the potential against the Fourier multiplier
    # -i D(k): equal in exact arithmetic, so only rounding separates them
    w = synth.Workload(f"fd{n}", n, n // 2, 2.0 * n, 0.3, 3, 4, 16, prec)
    inp = make_inputs(w)
    a = gpu_kick(w, inp)
    b = gpu_kick(w, inp, flags=KEEP_DEPOSIT | SPECTRAL_GRADIENT)
    emax, erms = force_errors(a["acc"], b["acc"])
    print(f"{prec} N={n}: stencil vs multiplier max {emax:.2e} rms {erms:.2e} (of rms |F|)")
    if prec == "fp64":
        assert emax < 1e-10
    else:   # FP32 differences of the potential: cancellation bounded by eps * phi / (d |grad phi|)
        assert erms < 3e-5


@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp32", 64)])
def test_prepared_response_is_identical(prec, n):
    # pm_nu_prepare runs the history panels on the side stream ahead of the
    # deposit: the response that joins them is bit-identical to one without,
    # and a prepare at another a makes the response recompute them
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"prep{n}", ngrid=n, npart_side=n, precision=prec,
                    n_hist=10)
    inp = make_inputs(w)
    a = gpu_kick(w, inp)
    b = gpu_kick(w, inp, prepare_a=w.a_kick)
    c = gpu_kick(w, inp, prepare_a=w.a_kick * 1.01)
    for key in ("R", "Pnu", "PM", "acc", "vel"):
        assert np.array_equal(a[key], b[key]), key
        assert np.array_equal(a[key], c[key]), key
    _check_common(w, b, oracle_kick(w, inp), prec == "fp64")


@pytest.mark.parametrize("prec,n,case", [("fp32", 64, "lattice"), ("fp64", 32, "lattice"), ("fp32", 64, "shuffled"),
                                         ("fp32", 64, "clustered"), ("fp32", 192, "lattice")])
def test_row_order_gather(prec, n, case):
    # gather_rows = 1 walks the deposit's row sort (records + permutation), 2
    # the same order writing forces by sorted slot and then the velocities in
    # particle order (inverse permutation): the same stencil arithmetic, so the
    # same forces and velocities bit for bit as the particle-order gather, for
    # lattice-ordered, shuffled and clustered particles; and against the oracle
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"rows{n}{case}", ngrid=n, npart_side=n // 2 if n > 32 else n,
                    precision=prec, n_hist=6, clustered=(case == "clustered"))
    inp = make_inputs(w)
    if case == "shuffled":
        perm = np.random.default_rng(3).permutation(inp["pos64"].shape[1])
        inp = dict(inp, pos64=inp["pos64"][:, perm].copy(), vel=inp["vel"][:, perm].copy())
    a = gpu_kick(w, inp, tuning=(-1, -1, 16, 0))
    b = gpu_kick(w, inp, tuning=(-1, -1, 16, 1))
    c = gpu_kick(w, inp, tuning=(-1, -1, 16, 2))
    assert np.array_equal(a["acc"], b["acc"])
    assert np.array_equal(a["vel"], b["vel"])
    assert np.array_equal(a["acc"], c["acc"])
    assert np.array_equal(a["vel"], c["vel"])
    _check_common(w, b, oracle_kick(w, inp), prec == "fp64")


def test_row_order_gather_needs_the_deposit_positions():
    # a kick with another position buffer than the deposit's falls back to the
    # particle-order gather (same results)
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="rowsfb", ngrid=64, npart_side=32, precision="fp32", n_hist=4)
    inp = make_inputs(w)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=4, precision="fp32",
                 sqrtPnu_init=inp["pi"], theta_over_delta_init=inp["ti"])
    pos = torch.from_numpy(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)).cuda()
    h = torch.from_numpy(np.ascontiguousarray(inp["hist"])).cuda()
    out = []
    for rows, other in ((0, False), (1, True), (1, False), (2, True), (2, False)):
        pm.set_tuning(-1, -1, 16, rows)
        vel = torch.from_numpy(inp["vel"].astype(np.float32)).cuda()
        acc = torch.empty_like(vel)
        pm.deposit(pos)
        pm.nu_response(w.a_kick, inp["a_hist"], h)
        pm.kick(pos.clone() if other else pos, vel, w.a_kick, 0.01, acc_out=acc)
        pm.check()
        out.append(acc.cpu().numpy())
    for o in out[1:]:
        assert np.array_equal(out[0], o)
    pm.close()


def test_forces_by_slot_leave_a_skipped_particle():
    # gather_rows = 2 with one particle whose offset is outside [0, 1): the sort
    # skips it (PM_ERR_RANGE), its velocity stays as it was, and every other
    # velocity equals the particle-order gather's
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name="rows2bad", ngrid=64, npart_side=32, precision="fp32",
                    n_hist=4)
    inp = make_inputs(w)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=4, precision="fp32",
                 sqrtPnu_init=inp["pi"], theta_over_delta_init=inp["ti"])
    bad = synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)
    bad[3, 5] = np.float32(1.0).view(np.int32)
    pos = torch.from_numpy(bad).cuda()
    h = torch.from_numpy(np.ascontiguousarray(inp["hist"])).cuda()
    v0 = inp["vel"].astype(np.float32)
    out = []
    for rows in (0, 2):
        pm.set_tuning(-1, -1, 16, rows)
        vel = torch.from_numpy(v0).cuda()
        pm.deposit(pos)
        pm.nu_response(w.a_kick, inp["a_hist"], h)
        pm.kick(pos, vel, w.a_kick, 0.01)
        with pytest.raises(nupm.PMError) as e:
            pm.check()
        assert e.value.code == -2                        # PM_ERR_RANGE
        out.append(vel.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[1][:, 5], v0[:, 5])
    assert not np.array_equal(out[1][:, 6], v0[:, 6])
    pm.close()


@pytest.mark.parametrize("flags", [KEEP_DEPOSIT, KEEP_DEPOSIT | UNFUSED_DEPOSIT])
def test_deposit_overflow_is_reported(flags):
    # a cell's fixed-point sum is an unsigned 64-bit integer and a particle at
    # a node gives it 2^48: 40000 particles there are deposited exactly
    # (40000 * 2^48 at the node, nothing elsewhere), 70000 pass 2^64 and
    # pm_check reports PM_ERR_OVERFLOW (fused tile sums and global sums)
    n = 32
    for npart, overflow in ((40000, False), (70000, True)):
        pos = np.zeros((6, npart), dtype=np.int32)
        pos[0:3] = 5                                          # cell (5, 5, 5), offsets 0
        pm = nupm.PM(n, npart, 64.0, 0.3, m_nu_total=0.0, a_init=0.02, n_kbins=8, precision="fp32", flags=flags)
        pm.deposit(torch.from_numpy(pos).cuda())
        if overflow:
            with pytest.raises(nupm.PMError) as e:
                pm.check()
            assert e.value.code == -3                        # PM_ERR_OVERFLOW
        else:
            pm.check()
            F = pm.field(nupm.FIELD_DEPOSIT).cpu().numpy().view(np.uint64).reshape(n, n, n)
            assert int(F[5, 5, 5]) == npart * 2 ** 48
            F[5, 5, 5] = 0
            assert not F.any()
        pm.close()


def test_prepare_twice_is_an_order_error():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], n_hist=4)
    inp = make_inputs(w)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=4, precision="fp64",
                 sqrtPnu_init=inp["pi"], theta_over_delta_init=inp["ti"])
    h = torch.from_numpy(np.ascontiguousarray(inp["hist"])).cuda()
    pm.nu_prepare(w.a_kick, inp["a_hist"], h)
    with pytest.raises(nupm.PMError) as e:
        pm.nu_prepare(w.a_kick, inp["a_hist"], h)
    assert e.value.code == -7
    pm.deposit(torch.from_numpy(inp["pos64"]).cuda())
    pm.nu_response(w.a_kick, inp["a_hist"], h)
    pm.check()
    pm.close()


def test_options_iters_fit_deconv_nohist_prev():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], n_hist=10)
    inp = make_inputs(w)
    prev = np.abs(inp["pi"][0]) * 1.7
    for kw, okw in ((dict(iters=2), dict(iters=2)),
                    (dict(flags=0x1 | KEEP_DEPOSIT), dict(I_func=O.nu_I_fit)),
                    (dict(flags=0x2 | KEEP_DEPOSIT), dict(deconvolve=True)),
                    (dict(n_hist=0), dict(n_hist=0)),
                    (dict(prev=prev), dict(prev=prev))):
        g = gpu_kick(w, inp, **kw)
        r = oracle_kick(w, inp, **okw)
        _check_common(w, g, r, True)


def test_massless_neutrinos_cdm_only():
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], m_nu_total=0.0, n_hist=4)
    inp = make_inputs(w)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    assert np.all(g["R"] == 0) and np.all(g["Pnu"] == 0)
    _check_common(w, g, r, True)


def test_single_particle_and_boundaries():
    # two particles: one in the last cell with offset 0 on x and just below 1
    # on z (wraps), one at a cell corner; forces compared on the scale of the
    # pair force at one cell, 1.5 Om L^3 / (4 pi a Delta^2)
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], n_hist=2)
    inp = make_inputs(w)
    L, n = w.box, w.ngrid
    d = L / n
    pos = np.array([[(n - 1) * d, 3 * d], [0.0, 7 * d], [L - 1e-9, 11 * d]])
    two = dict(inp, pos64=pos, vel=np.zeros((3, 2)))
    g = gpu_kick(w, two)
    r = oracle_kick(w, two)
    assert np.array_equal(g["F"].astype(np.int64), r.F)
    scale = 1.5 * w.omega_m * L ** 3 / (4 * math.pi * w.a_kick * d * d)
    assert np.max(np.abs(g["acc"] - r.acc)) < 1e-11 * scale
    assert np.max(np.abs(r.acc)) > 1e-6 * scale            # the pair force is resolved


def test_errors_reported():
    from paper_1209_0461_gb300 import nupm
    w = synth.WORKLOADS["pm32_fp64"]
    inp = make_inputs(w)
    dev = torch.device("cuda")
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, 3,
                 a_init=w.a_init, n_kbins=w.n_kbins, precision="fp32")
    cells = synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)
    bad = cells.copy()
    bad[3, 5] = np.float32(1.0).view(np.int32)          # offset outside [0, 1)
    pos = torch.from_numpy(bad).to(dev).contiguous()
    vel = torch.zeros((3, w.npart), dtype=torch.float32, device=dev)
    with pytest.raises(nupm.PMError) as e:
        pm.kick(pos, vel, w.a_kick, 0.01)
    assert e.value.code == -7                            # PM_ERR_ORDER
    pm.deposit(pos)
    with pytest.raises(nupm.PMError) as e:
        pm.check()
    assert e.value.code == -2                            # PM_ERR_RANGE
    pm.check()                                           # cleared
    with pytest.raises(nupm.PMError) as e:
        pm.nu_response(0.5 * w.a_init, [], None)
    assert e.value.code == -2
    with pytest.raises(nupm.PMError) as e:
        pm.nu_response(w.a_kick, [w.a_kick * 2], torch.zeros((1, w.n_kbins), dtype=torch.float64,
                                                             device=dev))
    assert e.value.code == -2
    pm.nu_response(w.a_kick, [], None)
    with pytest.raises(nupm.PMError) as e:
        pm.kick(pos, vel, w.a_kick * 1.01, 0.01)
    assert e.value.code == -7
    pm.close()


def test_kick_and_drift_factors():
    from paper_1209_0461_gb300 import nupm
    w = synth.WORKLOADS["pm32_fp64"]
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, 3)
    for a0, a1 in ((0.02, 0.1), (0.1, 0.1003), (0.5, 1.0)):
        assert abs(pm.kick_factor(a0, a1) / O.kick_factor(a0, a1, w.omega_m) - 1) < 1e-13
        assert abs(pm.drift_factor(a0, a1) / O.drift_factor(a0, a1, w.omega_m) - 1) < 1e-13
    pm.close()
    eds = nupm.PM(32, 8, 64.0, 1.0, 0.0, 0.7, 0.0, 0)
    assert abs(eds.kick_factor(0.1, 0.4) - 2 / 3 * (0.4 ** 1.5 - 0.1 ** 1.5)) < 1e-14
    eds.close()


def test_deposit_deterministic_under_shuffle():
    w = synth.WORKLOADS["pm32_fp64"]
    inp = make_inputs(w)
    perm = np.random.default_rng(3).permutation(w.npart)
    shuf = dict(inp, pos64=inp["pos64"][:, perm].copy(), vel=inp["vel"][:, perm].copy())
    g1 = gpu_kick(w, inp)
    g2 = gpu_kick(w, shuf)
    g3 = gpu_kick(w, inp)
    assert np.array_equal(g1["F"], g2["F"]) and np.array_equal(g1["F"], g3["F"])
    assert np.allclose(g1["acc"][:, perm], g2["acc"], rtol=0, atol=1e-12 * np.abs(g1["acc"]).max())


@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp32", 64), ("fp32", 256), ("fp64", 128)])
def test_fused_deposit_equals_unfused(prec, n):
    # the row-sorted shared-memory deposit fused with the x transform gives the
    # same integer grid and the same spectrum as the global-atomic path, for
    # lattice-ordered and shuffled particles
    w = synth.Workload(f"fuse{n}", n, n // 2 if n > 64 else n, 2.0 * n, 0.06, 3, 4, 16, prec)
    inp = make_inputs(w)
    perm = np.random.default_rng(11).permutation(inp["pos64"].shape[1])
    shuf = dict(inp, pos64=inp["pos64"][:, perm].copy(), vel=inp["vel"][:, perm].copy())
    a = gpu_kick(w, inp, flags=UNFUSED_DEPOSIT)
    b = gpu_kick(w, inp, flags=KEEP_DEPOSIT)
    c = gpu_kick(w, shuf, flags=KEEP_DEPOSIT)
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["F"], c["F"])
    # fused and shuffled runs see the same integer tile: identical to each other
    assert np.array_equal(b["spec"], c["spec"])
    assert np.array_equal(b["acc"][:, perm], c["acc"])
    if prec == "fp64":          # exact integer -> double conversion on both paths
        assert np.array_equal(a["spec"], b["spec"])
    else:                       # FP32: the compiler may contract the two paths' conversions differently
        rms = np.sqrt(np.mean(np.abs(a["spec"]) ** 2))
        assert np.sqrt(np.mean(np.abs(a["spec"] - b["spec"]) ** 2)) < 1e-6 * rms
    _, erms = force_errors(b["acc"], a["acc"])
    assert erms < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp32", 64), ("fp32", 128), ("fp64", 64)])
def test_tma_column_passes_equal_plain(prec, n):
    # the TMA-pipelined column passes do the same arithmetic in the same order
    # as the plain column kernels: identical spectra and forces
    w = synth.Workload(f"tma{n}", n, n, 2.0 * n, 0.15, 3, 4, 16, prec)
    inp = make_inputs(w)
    a = gpu_kick(w, inp, flags=KEEP_DEPOSIT | 0x10)     # PM_TMA_COLUMNS (gradient in Fourier space)
    b = gpu_kick(w, inp, flags=KEEP_DEPOSIT | SPECTRAL_GRADIENT)
    assert np.array_equal(a["spec"], b["spec"])
    assert np.array_equal(a["acc"], b["acc"])


@pytest.mark.parametrize("prec,flags", [("fp32", KEEP_DEPOSIT), ("fp64", KEEP_DEPOSIT),
                                        ("fp32", KEEP_DEPOSIT | SPECTRAL_GRADIENT)])
def test_tma_staged_z_passes(prec, flags):
    # wide_z = 2: z passes whose 128-byte-segment tiles are staged by TMA in
    # the exchange buffer; against the oracle, and the same arithmetic as the
    # plain wide z kernels (Green pass with one output, or two with the
    # gradient in Fourier space)
    w = synth.Workload("tmaz256", 256, 40, 512.0, 0.15, 3, 4, 16, prec)
    inp = make_inputs(w)
    g = gpu_kick(w, inp, tuning=(-1, 2, 16), flags=flags)
    _check_common(w, g, oracle_kick(w, inp), prec == "fp64")
    b = gpu_kick(w, inp, tuning=(-1, 1, 16), flags=flags)
    assert np.array_equal(g["spec"], b["spec"])
    # the two kernels inline the same butterflies, but the compiler may fuse
    # their multiply-adds differently: potentials an ulp apart, which the
    # real-space stencil's differences amplify by about phi / (cell |grad phi|)
    # (~40 here)
    emax, erms = force_errors(g["acc"], b["acc"])
    if prec == "fp64":
        assert emax < 1e-12
    else:
        assert erms < (1e-6 if flags & SPECTRAL_GRADIENT else 1e-5)


@pytest.mark.parametrize("n,nk", [(256, 256), (512, 64), (1024, 256)])
def test_bin_sums_fused_in_the_z_pass(n, nk):
    # wide_z = 2 with FP32 and at most 256 bins: the forward z pass sums the
    # bins' power (rings along kz, the packed x2 = 0 column by its own
    # kernel); the same counts and Sigma |k| as the lattice, and the power
    # sums of the separate bin pass to float rounding, on the same deposit
    w = synth.Workload(f"zbins{n}", n, n // 4, 2.0 * n, 0.15, 3, 4, nk, "fp32")
    inp = make_inputs(w)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=nk, n_hist_max=4, precision="fp32")
    pos = torch.from_numpy(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)).cuda()
    out = []
    for wide_z in (1, 2, 2):
        pm.set_tuning(-1, wide_z, 16)
        pm.deposit(pos)
        pm.check()
        out.append([np.array(x) for x in pm.bins()])
    pm.close()
    (c1, k1, p1), (c2, k2, p2), (c3, k3, p3) = out
    assert np.array_equal(c1, c2) and np.array_equal(k1, k2)
    ne = c1 > 0
    rel = np.abs(p2[ne] / p1[ne] - 1)
    print(f"n={n} nk={nk}: fused vs separate bin sums, max rel {rel.max():.2e}")
    assert rel.max() < 2e-6
    assert np.array_equal(p2, p3)                         # deterministic


@pytest.mark.parametrize("prec,n,npart", [("fp64", 32, 32 ** 3), ("fp32", 64, 64 ** 3 - 37),
                                          ("fp32", 128, 64 ** 3), ("fp64", 16, 8 ** 3)])
def test_fused_interpolation_equals_separate(prec, n, npart):
    # sliding-window inverse x + interpolation (no force grids) against the
    # separate inverse x pass and gather: same forces and velocities
    side = round(npart ** (1 / 3)) + 1
    w = synth.Workload(f"xint{n}", n, min(side, n), 2.0 * n, 0.3, 3, 4, 16, prec)
    inp = make_inputs(w, npart=min(npart, w.npart))
    a = gpu_kick(w, inp, flags=KEEP_DEPOSIT | SPECTRAL_GRADIENT)
    b = gpu_kick(w, inp, flags=KEEP_DEPOSIT | FUSED_GATHER)
    scale = np.max(np.abs(a["acc"]))
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.max(np.abs(a["acc"] - b["acc"])) <= tol * scale
    assert np.max(np.abs(a["vel"] - b["vel"])) <= tol * np.max(np.abs(a["vel"])) + 1e-30


@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp32", 64)])
def test_hierarchy_kick_three_unequal_species(prec, n):
    # Sec. 6.2 / Table 1: the S03NH normal-hierarchy masses 0.022, 0.024,
    # 0.054 eV, each species with its own free-streaming initial condition,
    # summed with weights m_i / M_nu; per bin and per particle against the oracle
    w = synth.hierarchy(synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"nh{n}_{prec}", ngrid=n,
                                    npart_side=n, box=4.0 * n, precision=prec, n_hist=12, n_kbins=24))
    assert w.masses == synth.HIERARCHY_NH
    inp = make_inputs(w)
    assert not np.allclose(inp["pi"][0], inp["pi"][2])      # the species' ICs differ
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    _check_common(w, g, r, prec == "fp64")
    # the hierarchy is not the degenerate case of the same total mass
    wd = synth.with_(w, m_species=())
    rd = O.nu_response(r.bins["k"], np.sqrt(r.bins["P"]), w.a_kick, cosmo_of(wd), inp["a_hist"], inp["hist"],
                       *synth.nu_initial(wd), nonempty=r.bins["nonempty"])
    ne = r.bins["nonempty"]
    assert np.max(np.abs(rd["R"][ne] / r.response["R"][ne] - 1)) > 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ic_multipole_j1_form(prec):
    # PM_IC_MULTIPOLE: the initial-condition term by Eq. deltaI-multipole, its
    # l = 1 part from the momentum integral of j_1 on the GPU, against the
    # oracle's j_1 integral (QUADPACK); at the config-1 setup (a_i = 0.02 ->
    # 0.1, so the IC term still matters at low k) and with a history of 2 nodes
    w = synth.with_(synth.WORKLOADS["pm32_fp64"], name=f"mp_{prec}", precision=prec, n_hist=2,
                    ngrid=32 if prec == "fp64" else 64, npart_side=32 if prec == "fp64" else 64)
    inp = make_inputs(w)
    g = gpu_kick(w, inp, flags=KEEP_DEPOSIT | nupm.PM_IC_MULTIPOLE)
    g0 = gpu_kick(w, inp)
    cos = cosmo_of(w)
    if prec == "fp64":
        c, q = O.quantise_positions_f64(inp["pos64"], w.box, w.ngrid)
        vel = inp["vel"]
    else:
        cell, off = synth.split_cell_offset(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid))
        c, q = O.quantise_positions_cell(cell, off, w.ngrid)
        vel = inp["vel"].astype(np.float32).astype(np.float64)
    F = O.cic_deposit(c, q, w.ngrid)
    spec = O.forward_fft(O.density_contrast(F, c.shape[1]))
    b = O.bin_power(spec, w.box, w.n_kbins)
    a_hist, hist = inp["a_hist"][:2], inp["hist"][:2]
    ref = O.nu_response(b["k"], np.sqrt(b["P"]), w.a_kick, cos, a_hist, hist, inp["pi"], inp["ti"],
                        nonempty=b["nonempty"], multipole=True)
    ne = b["nonempty"]
    rel = np.abs(g["R"][ne] / ref["R"][ne] - 1)
    diff = np.abs(g["R"][ne] / g0["R"][ne] - 1)
    print(f"{prec}: j_1 form vs oracle max rel {rel.max():.2e}; vs the Eq. deltaI-nu form {diff.max():.2e}")
    assert rel.max() < (1e-9 if prec == "fp64" else 1e-5)
    assert diff.max() < 1e-9
