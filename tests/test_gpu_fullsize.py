"""Parity at the full benchmark size: a 1024^3 grid, 512^3 particles, FP32,
in the launch configuration the benchmark times (default flags, autotuned
tiles).  The oracle cannot run the whole kick at this size, so it computes
outputs one at a time from the particles:

  * the fixed-point deposit at sampled nodes (bit-exact), and its total mass;
  * delta_k at every mode of the lowest |k| bins and at random modes (up to
    the Nyquist planes);
  * those bins' mode counts, |k| sums and power sums, and their neutrino
    response (Eq. P-final) from the oracle's own P_cdm;
  * the potential phi_k (Eq. Poisson with the neutrino-corrected delta_M) at
    the modes those bins bracket, from the DFT of the kick's potential grid;

and checks properties that hold at any size: the CIC gather of an
antisymmetric stencil conserves momentum (sum_p acc_p = 0), and the kick
adds acc K to every velocity.  The per-particle FP32 forces are compared with
the FP64 kick of the same particles (FP64 positions, grids and transforms),
which the oracle checks element by element at every smaller size."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib, cosmo_of  # noqa: E402
from oracle import pm_oracle as O  # noqa: E402
from paper_1209_0461_gb300 import nupm, synth  # noqa: E402

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["pm1024_p512_fp32"]
N2_LIM = 13          # every mode with 0 < n^2 < 13 is enumerated


def _low_modes(n):
    r = math.isqrt(N2_LIM) + 1
    kz, ky, kx = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), np.arange(0, r + 1), indexing="ij")
    kz, ky, kx = kz.ravel(), ky.ravel(), kx.ravel()
    n2 = kz * kz + ky * ky + kx * kx
    keep = (n2 > 0) & (n2 < N2_LIM)
    # the half spectrum holds kx = 0 modes with both signs of (ky, kz)
    return kz[keep], ky[keep], kx[keep]


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()
    w = W
    n = w.ngrid
    parts = synth.particles(w)
    packed = synth.to_cell_offset(parts["pos64"], w.box, n)
    pos64_h = parts.pop("pos64")
    vel64_h = parts.pop("vel")
    vel_h = vel64_h.astype(np.float32)
    a_hist, hist = synth.history(w)
    pi, ti = synth.nu_initial(w)
    dev = torch.device("cuda")
    pos = torch.from_numpy(packed).to(dev)
    vel = torch.from_numpy(vel_h).to(dev)
    hist_d = torch.from_numpy(np.ascontiguousarray(hist)).to(dev)
    nk = w.n_kbins
    a = w.a_kick
    out = {}
    # the benchmark's context: default flags, autotuned tiles
    pm = nupm.PM(n, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=nk, n_hist_max=w.n_hist, precision="fp32",
                 sqrtPnu_init=pi, theta_over_delta_init=ti, flags=0)
    K = pm.kick_factor(a, a * 1.01)
    vel_t = vel.clone()
    out["tuning"] = pm.autotune(pos, vel_t, a, a_hist, hist_d, reps=1)
    R = torch.zeros(nk, dtype=torch.float64, device=dev)
    Pn = torch.zeros_like(R)
    PM_ = torch.zeros_like(R)
    acc = torch.empty_like(vel)
    vel_t = vel.clone()
    pm.deposit(pos)
    pm.nu_response(a, a_hist, hist_d, None, R, Pn, PM_)
    spec = pm.field(nupm.FIELD_DELTA_K)
    lz, ly, lx = _low_modes(n)
    rng = np.random.default_rng(1234)
    hz = np.concatenate([rng.integers(-n // 2, n // 2, 5), [0, -n // 2, 7]])
    hy = np.concatenate([rng.integers(-n // 2, n // 2, 5), [-n // 2, 0, -n // 2]])
    hx = np.concatenate([rng.integers(1, n // 2, 5), [n // 2, 3, n // 2]])
    take = lambda z, y, x: spec[torch.from_numpy(np.mod(z, n)).to(dev), torch.from_numpy(np.mod(y, n)).to(dev),
                                torch.from_numpy(x).to(dev)].cpu().numpy()
    out["low"] = (lz, ly, lx, take(lz, ly, lx))
    out["high"] = (hz, hy, hx, take(hz, hy, hx))
    del spec
    out["bins"] = pm.bins()
    out["R"], out["Pnu"], out["PM"] = R.cpu().numpy(), Pn.cpu().numpy(), PM_.cpu().numpy()
    pm.kick(pos, vel_t, a, K, acc_out=acc)
    pm.check()
    out["K"] = K
    out["acc_sum"] = acc.double().sum(dim=1).cpu().numpy()
    out["acc_abs"] = acc.double().abs().sum(dim=1).cpu().numpy()
    fidx = torch.from_numpy(np.sort(rng.choice(w.npart, 1 << 17, replace=False))).to(dev)
    out["acc32_f"] = acc[:, fidx].double().cpu().numpy()
    sidx = torch.from_numpy(rng.integers(0, w.npart, 4096)).to(dev)
    out["v_new"] = vel_t[:, sidx].double().cpu().numpy()
    out["dv"] = (vel_t[:, sidx].double() - vel[:, sidx].double()).cpu().numpy()
    out["acc_s"] = acc[:, sidx].double().cpu().numpy()
    del acc, vel_t
    # potential grid: DFT at the low modes (float64 slabs on the device)
    phi = pm.field(nupm.FIELD_PHI)
    x = torch.arange(n, dtype=torch.float64, device=dev)
    uz, iz_of = np.unique(lz, return_inverse=True)
    uy, iy_of = np.unique(ly, return_inverse=True)
    ux, ix_of = np.unique(lx, return_inverse=True)
    E = lambda u: torch.exp(-2j * math.pi * torch.outer(x, torch.from_numpy(u).to(dev).double()) / n)
    Ex, Ey, Ez = E(ux), E(uy), E(uz)
    D = torch.zeros((uz.size, uy.size, ux.size), dtype=torch.complex128, device=dev)
    for z0 in range(0, n, 64):
        A = phi[z0:z0 + 64].double()
        B = torch.complex(A @ Ex.real, A @ Ex.imag)             # [z, y, kx]
        C = torch.einsum("zyk,yj->zjk", B, Ey)
        D += torch.einsum("zjk,zl->ljk", C, Ez[z0:z0 + 64])
    out["phi_low"] = D.cpu().numpy()[iz_of, iy_of, ix_of]
    del phi
    pm.close()
    # the same deposit, kept: the fixed-point grid at sampled nodes and its total
    pmk = nupm.PM(n, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                  a_init=w.a_init, n_kbins=nk, n_hist_max=w.n_hist, precision="fp32",
                  sqrtPnu_init=pi, theta_over_delta_init=ti, flags=nupm.PM_KEEP_DEPOSIT)
    pmk.deposit(pos)
    F = pmk.field(nupm.FIELD_DEPOSIT).view(-1)
    cells = np.concatenate([[0, n ** 3 - 1, n - 1, (n - 1) * n, (n - 1) * n * n],
                            rng.integers(0, n ** 3, 59)]).astype(np.int64)
    out["cells"] = cells
    out["F_cells"] = F[torch.from_numpy(cells).to(dev)].cpu().numpy()
    rows = F.view(n * n, n).sum(dim=1).cpu().numpy()        # each row sum < 2^63
    out["F_total"] = sum(int(v) for v in rows.tolist())
    del F
    pmk.close()
    # the FP64 kick of the same particles (FP64 positions), same response inputs
    del pos, vel
    torch.cuda.empty_cache()
    pm64 = nupm.PM(n, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                   a_init=w.a_init, n_kbins=nk, n_hist_max=w.n_hist, precision="fp64",
                   sqrtPnu_init=pi, theta_over_delta_init=ti, flags=0)
    p64 = torch.from_numpy(pos64_h).to(dev)
    v64 = torch.from_numpy(vel64_h).to(dev)
    a64 = torch.empty_like(v64)
    pm64.deposit(p64)
    pm64.nu_response(a, a_hist, hist_d)
    pm64.kick(p64, v64, a, K, acc_out=a64)
    pm64.check()
    out["acc64_f"] = a64[:, fidx].cpu().numpy()
    out["acc64_rms"] = float(torch.sqrt((a64 * a64).sum(dim=0).mean()).item())
    del p64, v64, a64
    pm64.close()
    # oracle inputs: the same seeded particles, quantised by the oracle
    cell, off = synth.split_cell_offset(packed)
    c, q = O.quantise_positions_cell(cell, off, n)
    out["c"], out["q"] = c, q
    out["inputs"] = dict(a_hist=a_hist, hist=hist, pi=pi, ti=ti)
    return out


def test_deposit_at_sampled_nodes_and_total_mass(run):
    ref = O.cic_deposit_cells(run["c"], run["q"], W.ngrid, run["cells"])
    assert np.array_equal(run["F_cells"].astype(np.int64), ref)
    assert run["F_total"] == W.npart * 2 ** 48


def _oracle_low(run):
    if "oracle_low" not in run:
        lz, ly, lx, _ = run["low"]
        dk = O.density_modes(run["c"], run["q"], W.ngrid, W.npart, lz, ly, lx)
        b = O.bin_power_modes(dk, lz, ly, lx, W.ngrid, W.box, W.n_kbins)
        run["oracle_low"] = (dk, b)
    return run["oracle_low"]


def test_spectrum_at_low_and_random_modes(run):
    dk, _ = _oracle_low(run)
    got = run["low"][3]
    rel = np.abs(got - dk) / np.abs(dk)
    print(f"low modes: {dk.size}, max rel {rel.max():.2e}")
    assert rel.max() < 2e-5
    hz, hy, hx, goth = run["high"]
    refh = O.density_modes(run["c"], run["q"], W.ngrid, W.npart, hz, hy, hx)
    scale = np.sqrt(np.mean(np.abs(refh) ** 2))
    err = np.abs(goth - refh) / scale
    print(f"random modes: max |d| / rms {err.max():.2e}")
    assert err.max() < 2e-5


def _complete_bins(b):
    T = b["T"]
    done = (T[1:] <= N2_LIM) & b["nonempty"]
    assert done.sum() >= 5
    return done


def test_low_bins_and_their_response(run):
    dk, b = _oracle_low(run)
    done = _complete_bins(b)
    cnt, ks, ps = run["bins"]
    assert np.array_equal(cnt[done], b["count"][done])
    assert np.allclose(ks[done], b["ksum"][done], rtol=1e-12, atol=0)
    assert np.allclose(ps[done], b["psum"][done], rtol=4e-5, atol=0)
    inp = run["inputs"]
    sel = np.nonzero(done)[0]
    ref = O.nu_response(b["k"][sel], np.sqrt(b["P"][sel]), W.a_kick, cosmo_of(W), inp["a_hist"],
                        inp["hist"][:, sel], inp["pi"][:, sel], inp["ti"][:, sel])
    for key, got in (("R", run["R"]), ("sqrtPnu", run["Pnu"]), ("sqrtPM", run["PM"])):
        rel = np.abs(got[sel] - ref[key]) / np.abs(ref[key])
        assert rel.max() < 2e-5, (key, rel.max())


def test_potential_at_bracketed_modes(run):
    dk, b = _oracle_low(run)
    done = _complete_bins(b)
    lz, ly, lx, _ = run["low"]
    kf = 2.0 * math.pi / W.box
    kmag = kf * np.sqrt((lz * lz + ly * ly + lx * lx).astype(np.float64))
    kb, R = b["k"][done], run_R_oracle(run, b, done)
    inside = (kmag >= kb.min() * (1 - 1e-12)) & (kmag <= kb.max() * (1 + 1e-12))
    assert inside.sum() >= 20
    ref = O.potential_spectrum(dk[inside], W.box, W.a_kick, cosmo_of(W), kb, R, np.ones(kb.size, bool),
                               modes=(lz[inside], ly[inside], lx[inside]), ngrid=W.ngrid)
    got = run["phi_low"][inside]
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"potential at {inside.sum()} modes: max rel {rel.max():.2e}")
    assert rel.max() < 1e-4


def run_R_oracle(run, b, done):
    inp = run["inputs"]
    sel = np.nonzero(done)[0]
    return O.nu_response(b["k"][sel], np.sqrt(b["P"][sel]), W.a_kick, cosmo_of(W), inp["a_hist"],
                         inp["hist"][:, sel], inp["pi"][:, sel], inp["ti"][:, sel])["R"]


def test_momentum_conservation_and_kick(run):
    # sum_p acc_p = sum_x rho(x) (-S phi)(x) = 0: the gather is the deposit's
    # adjoint and the stencil composed with the even Green function is odd
    ratio = np.abs(run["acc_sum"]) / run["acc_abs"]
    print(f"|sum acc| / sum |acc| per axis: {ratio}")
    assert np.all(ratio < 1e-6)
    # u_new = u + acc K in FP32: one rounding of the result, K itself rounded
    # to FP32, at most one more of the product
    dv, acc = run["dv"], run["acc_s"]
    bound = 1.5e-7 * (np.abs(run["v_new"]) + np.abs(acc * run["K"])) + 1e-30
    assert np.all(np.abs(dv - acc * run["K"]) <= bound)
    assert np.max(np.abs(dv)) > 0


def test_fp32_forces_against_the_fp64_kick(run):
    # 2^17 sampled particles of the 1024^3 / 512^3 kick: FP32 (int32 cell +
    # FP32 offset positions, FP32 grids) against the FP64 kick
    a32, a64 = run["acc32_f"], run["acc64_f"]
    d = np.sqrt(((a32 - a64) ** 2).sum(0))
    rms = run["acc64_rms"]
    erms, emax = float(np.sqrt((d ** 2).mean()) / rms), float(d.max() / rms)
    print(f"FP32 vs FP64 forces at 1024^3: rms {erms:.2e}, max {emax:.2e} of the rms force")
    assert erms < 2e-4
    assert emax < 2e-3
