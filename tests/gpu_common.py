"""Shared helpers of the GPU parity tests: run one kick through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np

from oracle import pm_oracle as O
from paper_1209_0461_gb300 import nupm, synth


def build_lib():
    from paper_1209_0461_gb300 import build as b
    b.build()
    return nupm.lib()


def cosmo_of(w):
    return O.Cosmo(w.omega_cdm, w.omega_nu, w.h, w.masses, w.a_init)


def make_inputs(w, npart=None, seed_shift=0):
    """Particles, history and ICs of workload w; optionally drop particles to
    a ragged count."""
    import torch
    parts = synth.particles(synth.with_(w, seed=w.seed + seed_shift))
    pos64, vel = parts["pos64"], parts["vel"]
    if npart is not None:
        pos64, vel = pos64[:, :npart].copy(), vel[:, :npart].copy()
    a_hist, hist = synth.history(w)
    pi, ti = synth.nu_initial(w)
    return dict(pos64=pos64, vel=vel, a_hist=a_hist, hist=hist, pi=pi, ti=ti)


KEEP_DEPOSIT = 0x4
UNFUSED_DEPOSIT = 0x8
FUSED_GATHER = 0x20
SPECTRAL_GRADIENT = 0x40


def gpu_kick(w, inp, K=0.01, iters=1, flags=KEEP_DEPOSIT, n_hist=None, prev=None, quad=8, keep_fields=False,
             tuning=None, prepare_a=None):
    """Deposit, response and kick through the C ABI (tuning: pm_set_tuning
    knobs, or None for the built-in choices; prepare_a: call pm_nu_prepare at
    that scale factor before the deposit).  Returns numpy results."""
    import torch
    dev = torch.device("cuda")
    fp64 = w.precision == "fp64"
    np_ = inp["pos64"].shape[1]
    a_hist, hist = inp["a_hist"], inp["hist"]
    if n_hist is not None:
        a_hist, hist = a_hist[:n_hist], hist[:n_hist]
    pm = nupm.PM(w.ngrid, np_, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 m_nu=w.m_species or None,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=max(len(a_hist), 1),
                 precision=w.precision, flags=flags, iters=iters, quad_nodes=quad,
                 sqrtPnu_init=inp["pi"], theta_over_delta_init=inp["ti"])
    if tuning is not None:
        pm.set_tuning(*tuning)
    if fp64:
        pos = torch.from_numpy(inp["pos64"]).to(dev).contiguous()
        vel = torch.from_numpy(inp["vel"]).to(dev).contiguous()
    else:
        pos = torch.from_numpy(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid)).to(dev).contiguous()
        vel = torch.from_numpy(inp["vel"].astype(np.float32)).to(dev).contiguous()
    vel0 = vel.clone()
    acc = torch.empty_like(vel)
    hist_t = torch.from_numpy(np.ascontiguousarray(hist)).to(dev) if len(a_hist) else None
    if prepare_a is not None:
        pm.nu_prepare(prepare_a, a_hist, hist_t)
    pm.deposit(pos)
    F = pm.field(nupm.FIELD_DEPOSIT).cpu().numpy().view(np.uint64)
    spec = pm.field(nupm.FIELD_DELTA_K).cpu().numpy()
    nk = w.n_kbins
    R = torch.zeros(nk, dtype=torch.float64, device=dev)
    Pn = torch.zeros_like(R)
    PM_ = torch.zeros_like(R)
    prev_t = None if prev is None else torch.from_numpy(np.asarray(prev, dtype=np.float64)).to(dev)
    pm.nu_response(w.a_kick, a_hist, hist_t, prev_t, R, Pn, PM_)
    pm.kick(pos, vel, w.a_kick, K, acc_out=acc)
    pm.check()
    out = dict(F=F, spec=spec, R=R.cpu().numpy(), Pnu=Pn.cpu().numpy(), PM=PM_.cpu().numpy(),
               acc=acc.cpu().numpy().astype(np.float64), vel=vel.cpu().numpy().astype(np.float64),
               vel0=vel0.cpu().numpy().astype(np.float64), bins=pm.bins(), T=pm.thresholds(),
               pos=pos)
    if keep_fields:
        out["fields"] = [pm.field(nupm.FIELD_ACC_X + c).cpu().numpy() for c in range(3)]
        if not flags & (SPECTRAL_GRADIENT | FUSED_GATHER | 0x10):   # real-space gradient: the potential grid
            out["phi"] = pm.field(nupm.FIELD_PHI).cpu().numpy()
    pm.close()
    return out


def oracle_kick(w, inp, K=0.01, iters=1, deconvolve=False, I_func=O.nu_I, n_hist=None, prev=None):
    a_hist, hist = inp["a_hist"], inp["hist"]
    if n_hist is not None:
        a_hist, hist = a_hist[:n_hist], hist[:n_hist]
    if w.precision == "fp64":
        c, q = O.quantise_positions_f64(inp["pos64"], w.box, w.ngrid)
    else:
        cell, off = synth.split_cell_offset(synth.to_cell_offset(inp["pos64"], w.box, w.ngrid))
        c, q = O.quantise_positions_cell(cell, off, w.ngrid)
    vel = inp["vel"] if w.precision == "fp64" else inp["vel"].astype(np.float32).astype(np.float64)
    return O.pm_kick(c, q, vel, w.ngrid, w.box, w.a_kick, K, cosmo_of(w), w.n_kbins, a_hist, hist,
                     inp["pi"], inp["ti"], sqrtPnu_prev=prev, iters=iters, deconvolve=deconvolve,
                     I_func=I_func, keep_fields=True)


def force_errors(acc, ref):
    """(max |dF| / rms |F|, rms |dF| / rms |F|) over particles."""
    d = np.sqrt(((acc - ref) ** 2).sum(0))
    rms = np.sqrt((ref ** 2).sum(0).mean())
    return float(d.max() / rms), float(np.sqrt((d ** 2).mean()) / rms)
