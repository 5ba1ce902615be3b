#!/usr/bin/env python3
"""Benchmark of the GB300 PM kick with linear-response neutrinos.

metric: particle-kicks/s including the neutrino response, N_p / t(kick),
one kick = pm_deposit + pm_nu_response + pm_kick (CIC deposit, forward FFT,
P_cdm bins, FP64 response integral, Green/gradient, 3 inverse FFTs, CIC
interpolation and velocity update).

Default workload: the precision form, 512^3 particles (int32 cell + FP32
offset) on a 1024^3 FP32 grid, box 1 Gpc/h, M_nu = 0.06 eV (3 degenerate),
256 log-k bins, 128-step FP64 history; seeded BBKS Gaussian field,
Zel'dovich particles at a = 0.1 (synthetic stand-in for CAMB/N-GenICs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 runs under torchrun: independent boxes (seed + rank) per GPU, no
collective on the data path ("replicas only"), max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1209_0461_gb300 import synth  # noqa: E402

FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for i, nm in enumerate(names):
                if f[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def bins_in_z(w, tuning):
    """True when the FP32 bin power sums ride in the TMA-staged forward z pass
    (wide_z = 2 on a power-of-two grid of 256 or more, at most 256 bins): the
    bins stage then reads only the packed x2 = 0 column."""
    n = w.ngrid
    return (bool(tuning) and tuning[1] == 2 and w.precision == "fp32" and w.n_kbins <= 256
            and n >= 256 and (n & (n - 1)) == 0)


def stage_bytes(w, stage, fused_interp=True, spectral=False, bins_fused=False):
    """Algorithmic (compulsory) HBM bytes of ONE launch of a stage: each pass
    reads its inputs and writes its outputs once at stored precision.  By
    default the inverse passes carry the potential alone and the gather reads
    the real potential grid (its 4-point stencil); with the gradient in
    Fourier space (spectral) they carry three force fields.  With the fused
    interpolation the inverse x stage reads the three fields and the
    particles (positions, row permutation) and updates the velocities.  With
    the bin sums in the forward z pass (bins_fused) the bins stage reads the
    packed x2 = 0 column alone."""
    if bins_fused and stage == "bins":
        return (8 if w.precision == "fp32" else 16) * w.ngrid * w.ngrid
    n = w.ngrid
    M = n ** 3
    Mc = n * n * (n // 2)                 # packed complex elements per field
    r = 4 if w.precision == "fp32" else 8
    c = 2 * r
    p = 24                                 # position bytes per particle (both forms)
    v = r
    Np = w.npart
    if not (spectral or fused_interp):
        return {
            "deposit": (p + 8) * Np,
            "fft_x_fwd": 8 * Np + c * Mc,
            "fft_y_fwd": 2 * c * Mc,
            "fft_z_fwd": 2 * c * Mc,
            "bins": c * Mc,
            "green": 3 * c * n * n,
            "fft_z_inv": 2 * c * Mc,                      # spectrum -> phi
            "fft_y_inv": 2 * c * Mc,                      # phi in place
            "fft_x_inv": c * Mc + r * M,                  # packed rows -> real potential
            "interp": p * Np + min(r * M, 56 * r * Np) + 2 * 3 * v * Np,
            "drift": 2 * p * Np + 3 * v * Np,
        }.get(stage)
    return {
        "deposit": (p + 8) * Np,                         # row sort: positions in, 8-byte records out
        "fft_x_fwd": 8 * Np + c * Mc,                    # fused deposit + x: records in, spectrum out
        "fft_y_fwd": 2 * c * Mc,
        "fft_z_fwd": 2 * c * Mc,
        "bins": c * Mc,
        "green": 3 * c * n * n,                           # packed kx=0 plane: 2 reads + 1 write
        "fft_z_inv": c * Mc + 2 * c * Mc,                 # spectrum -> phi, d/dz phi
        "fft_y_inv": 2 * c * Mc + 3 * c * Mc,             # 2 fields -> 3 fields
        "fft_x_inv": (3 * c * Mc + (p + 4 + 2 * 3 * v) * Np) if fused_interp else 3 * (c * Mc + r * M),
        "interp": p * Np + min(3 * r * M, 24 * r * Np) + 2 * 3 * v * Np,
        "drift": 2 * p * Np + 3 * v * Np,                # positions read and written, velocities read
    }.get(stage)


def traffic_from_profiles(stage, workload):
    """DRAM bytes per launch of `stage` from the committed ncu summary, if it
    was taken on the current kernel sources (source hash recorded there)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for ln in open(path):
        f = ln.split()
        if len(f) >= 4 and f[0] == workload and f[1] == stage and f[2] == want:
            return float(f[3])
    return None


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1209_0461_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ oracle baseline
def oracle_sample(w, seed_shift=0):
    """A bounded CPU sample of the workload: same cosmology, bins, history and
    particle:grid ratio, on a 128^3 grid with 64^3 particles (cell size kept)."""
    scale = 128 / w.ngrid
    s = synth.with_(w, name=w.name + "_sample", ngrid=128, npart_side=max(8, int(w.npart_side * scale)),
                    box=w.box * scale, seed=w.seed + seed_shift)
    return s


def run_oracle_kick(s):
    from oracle import pm_oracle as O
    p = synth.particles(s)
    ah, hh = synth.history(s)
    pi, ti = synth.nu_initial(s)
    cos = O.Cosmo(s.omega_cdm, s.omega_nu, s.h, s.masses, s.a_init)
    if s.precision == "fp32":
        cell, off = synth.split_cell_offset(synth.to_cell_offset(p["pos64"], s.box, s.ngrid))
        c, q = O.quantise_positions_cell(cell, off, s.ngrid)
    else:
        c, q = O.quantise_positions_f64(p["pos64"], s.box, s.ngrid)
    t0 = time.perf_counter()
    O.pm_kick(c, q, p["vel"], s.ngrid, s.box, s.a_kick, 0.01, cos, s.n_kbins, ah, hh, pi, ti)
    return time.perf_counter() - t0, s.npart


def host_info():
    """CPU model and logical core count of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "hardware", "cpu model"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return model or "unknown", os.cpu_count() or 1


def _oracle_task(args):
    """One oracle kick of the bounded sample in a worker process; returns
    (particles, wall-clock start, end) of the kick itself."""
    name, shift = args
    w = synth.WORKLOADS[name]
    s = oracle_sample(w, seed_shift=shift)
    from oracle import pm_oracle as O
    p = synth.particles(s)
    ah, hh = synth.history(s)
    pi, ti = synth.nu_initial(s)
    cos = O.Cosmo(s.omega_cdm, s.omega_nu, s.h, s.masses, s.a_init)
    cell, off = synth.split_cell_offset(synth.to_cell_offset(p["pos64"], s.box, s.ngrid))
    c, q = (O.quantise_positions_cell(cell, off, s.ngrid) if s.precision == "fp32"
            else O.quantise_positions_f64(p["pos64"], s.box, s.ngrid))
    t0 = time.time()
    O.pm_kick(c, q, p["vel"], s.ngrid, s.box, s.a_kick, 0.01, cos, s.n_kbins, ah, hh, pi, ti)
    return s.npart, t0, time.time()


class OracleCores:
    """The oracle on every host core: one independent sample kick per core
    (spawned worker processes, started before any GPU work is timed)."""

    def __init__(self, workload_name, cores=None):
        import multiprocessing as mp
        self.name = workload_name
        self.cores = cores or (os.cpu_count() or 1)
        env = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
        os.environ.update(env)
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.step = 0

    def run(self):
        """Particle-kicks/s of one concurrent round (each core one kick)."""
        res = self.pool.map(_oracle_task, [(self.name, 1000 * self.step + i) for i in range(self.cores)])
        self.step += 1
        n = sum(r[0] for r in res)
        wall = max(r[2] for r in res) - min(r[1] for r in res)
        return n / wall, wall

    def close(self):
        self.pool.close()
        self.pool.join()


# ------------------------------------------------------------------ GPU arm
def replica(w, rank):
    """The box rank r runs: the same workload with seed + r (replicas only:
    boxes are independent, no collective on the data path)."""
    return synth.with_(w, seed=w.seed + rank)


def max_over_ranks(x, world, device=None):
    """The slowest rank's value (the job's time); x itself with one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units all ranks processed per second, timed by the slowest rank."""
    return world * units_per_rank / (ms_max / 1e3)


def run_gpu(args, w, rank, world):
    import torch
    from paper_1209_0461_gb300 import build as b
    from paper_1209_0461_gb300 import nupm
    b.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    torch.cuda.set_stream(torch.cuda.Stream(dev))   # a capturable stream for the context and the timing
    wr = replica(w, rank)
    t0 = time.time()
    parts = synth.particles(wr)
    a_hist, hist = synth.history(wr)
    pi, ti = synth.nu_initial(wr)
    fp32 = wr.precision == "fp32"
    if fp32:
        pos_h = torch.from_numpy(synth.to_cell_offset(parts["pos64"], wr.box, wr.ngrid))
        vel_h = torch.from_numpy(parts["vel"].astype(np.float32))
    else:
        pos_h = torch.from_numpy(parts["pos64"])
        vel_h = torch.from_numpy(parts["vel"])
    del parts
    pos_h, vel_h = pos_h.pin_memory(), vel_h.pin_memory()
    gen_s = time.time() - t0
    pos = pos_h.to(dev, non_blocking=True)
    vel = vel_h.to(dev, non_blocking=True)
    hist_d = torch.from_numpy(np.ascontiguousarray(hist)).to(dev)
    nk = wr.n_kbins
    out_R = torch.zeros(nk, dtype=torch.float64, device=dev)
    out_Pm = torch.zeros(nk, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    pm = nupm.PM(wr.ngrid, wr.npart, wr.box, wr.omega_cdm, wr.omega_nu, wr.h, wr.m_nu_total,
                 wr.n_species, a_init=wr.a_init, n_kbins=nk, n_hist_max=wr.n_hist,
                 precision=wr.precision, sqrtPnu_init=pi, theta_over_delta_init=ti, stream=stream,
                 flags=nupm.PM_SPECTRAL_GRADIENT if args.spectral_gradient else 0)
    a = wr.a_kick
    K = pm.kick_factor(a, a * 1.01)

    def step(p_, v_):
        # the response's history panels overlap the deposit on the context's side stream
        pm.nu_prepare(a, a_hist, hist_d)
        pm.deposit(p_)
        pm.nu_response(a, a_hist, hist_d, None, out_R, None, out_Pm)
        pm.kick(p_, v_, a, K)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    tuning = None
    if args.tuning:
        tuning = [int(v) for v in args.tuning.split(",")]
        pm.set_tuning(*tuning)
    elif not args.no_autotune:
        # kick factor 0 inside: velocities unchanged
        tuning = list(pm.autotune(pos, vel, a, a_hist, hist_d, reps=2))

    for _ in range(args.warmup):
        step(pos, vel)
    pm.check()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    pm.timing(True)
    with ClockSampler(dev.index) as clk:
        barrier()
        ev0.record(stream)
        for i in range(args.steps):
            evs[i].record(stream)
            step(pos, vel)
        evs[-1].record(stream)
        ev1.record(stream)
        barrier()
    stages = pm.get_timing()
    pm.timing(False)
    pm.check()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    ms_median = float(np.median([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]))
    # the same step captured once into a CUDA graph and replayed
    try:
        g = nupm.Graph.capture(stream, lambda: step(pos, vel))
        for _ in range(args.warmup):
            g.launch(stream)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            g.launch(stream)
        g1.record(stream)
        barrier()
        pm.check()
        msg = max_over_ranks(g0.elapsed_time(g1) / args.steps, world, dev)
        graph = {"ms_per_step": round(msg, 4), "value": whole_job_rate(wr.npart, world, msg), "nodes": g.nodes()}
        g.close()
    except nupm.PMError as e:
        graph = {"unavailable": str(e)}
    # end to end through the same API with host buffers: every step copies its
    # positions and velocities in from pinned host memory, kicks, and copies the
    # velocities out.  Copies run on their own streams with three device buffer
    # pairs, so step i+1's inputs travel while step i kicks and step i-1's
    # velocities travel out (with two pairs, step i+1's inputs would wait for
    # step i-1's output copy, which waits for its kick).
    e2e = None
    if not args.no_e2e:
        NBUF = 3
        vel_out = torch.empty_like(vel_h).pin_memory()
        # the inputs travel as 4 pieces on 4 streams
        h2d = [torch.cuda.Stream() for _ in range(4)]
        d2h = torch.cuda.Stream()
        bufs = [(pos, vel)] + [(torch.empty_like(pos), torch.empty_like(vel)) for _ in range(NBUF - 1)]
        ev_in = [[torch.cuda.Event() for _ in h2d] for _ in range(NBUF)]
        ev_done = [torch.cuda.Event() for _ in range(NBUF)]
        ev_out = [torch.cuda.Event() for _ in range(NBUF)]
        pieces_h = list(pos_h.view(-1).chunk(3)) + [vel_h.view(-1)]

        def e2e_steps(n):
            start = torch.cuda.Event()
            start.record(stream)                     # no copy starts before this point
            for hs in h2d:
                hs.wait_event(start)
            for i in range(n):
                b = i % NBUF
                p_, v_ = bufs[b]
                pieces_d = list(p_.view(-1).chunk(3)) + [v_.view(-1)]
                for hs, src, dst, ev in zip(h2d, pieces_h, pieces_d, ev_in[b]):
                    hs.wait_event(ev_out[b])         # buffer b's previous result is out
                    with torch.cuda.stream(hs):
                        dst.copy_(src, non_blocking=True)
                    ev.record(hs)
                    stream.wait_event(ev)
                step(p_, v_)
                ev_done[b].record(stream)
                d2h.wait_event(ev_done[b])
                with torch.cuda.stream(d2h):
                    vel_out.copy_(v_, non_blocking=True)
                ev_out[b].record(d2h)
            stream.wait_event(ev_out[(n - 1) % NBUF])

        e2e_steps(NBUF)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_steps(args.steps)
        e1.record(stream)
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        bi = pos_h.numel() * pos_h.element_size() + vel_h.numel() * vel_h.element_size()
        bo = vel_out.numel() * vel_out.element_size()
        e2e = {"value": whole_job_rate(wr.npart, world, ems), "unit": "particle-kicks/s",
               "ms_per_step": ems, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)}
    # roofline of the dominant kernel (largest total time among the HBM passes)
    hbm, peak_kind = peaks()
    cand = {k: v for k, v in stages.items() if k != "response" and v[1] > 0}
    dom = max(cand, key=lambda k: cand[k][0])
    tot_ms, launches, calls = stages[dom]
    per_launch_ms = tot_ms / max(launches, 1)
    if dom in ("deposit", "bins"):
        per_launch_ms = tot_ms / max(calls, 1)     # memset/reduce ride along in the stage
    fused = stages["interp"][1] == 0
    spectral = bool(args.spectral_gradient)
    bz = bins_in_z(wr, tuning)
    alg = stage_bytes(wr, dom, fused, spectral, bz)
    achieved = alg / (per_launch_ms / 1e3) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": traffic_from_profiles(dom, wr.name), "alg_bytes_per_launch": int(alg),
            "ms_per_launch": round(per_launch_ms, 4)}
    total_launch = sum(v[1] for v in stages.values())
    step_alg = sum(stage_bytes(wr, k, fused, spectral, bz) * (v[2] if k in ("deposit", "bins") else v[1])
                   for k, v in stages.items() if k != "response" and v[1] > 0) / args.steps
    res = dict(value=whole_job_rate(wr.npart, world, ms), ms_per_step=ms, ms_per_step_median=ms_median,
               graph=graph, e2e=e2e, roofline=roof,
               stages={k: {"ms_per_step": round(v[0] / args.steps, 4), "launches_per_step": v[1] // args.steps}
                       for k, v in stages.items()},
               gpu_launches=int(total_launch), clocks=clk.summary(), gen_s=round(gen_s, 1), tuning=tuning,
               step_alg_gb=round(step_alg / 1e9, 2),
               step_frac=round(step_alg / (ms / 1e3) / 1e9 / hbm, 4),
               device_bytes=pm.device_bytes())
    pm.close()
    return res


# ------------------------------------------------------------------ other forms
def _kick_form(w, pos64, vel64, precision, steps, warmup, mlp=None, keep_acc=True, stages_out=None,
               tuning_out=None, autotune=True):
    """Time `steps` kicks of workload w (inputs resident) in the given
    precision, exact or surrogate response, after pm_autotune (as the main
    measurement; the exact response's panels prepared beside the deposit).
    Returns (ms per kick, response ms per kick, acc [3, Np] on the device or None)."""
    import torch
    from paper_1209_0461_gb300 import nupm
    dev = torch.device("cuda")
    a_hist, hist = synth.history(w)
    pi, ti = synth.nu_initial(w)
    if precision == "fp32":
        pos = torch.from_numpy(synth.to_cell_offset(pos64, w.box, w.ngrid)).to(dev)
        vel = torch.from_numpy(vel64.astype(np.float32)).to(dev)
    else:
        pos = torch.from_numpy(pos64).to(dev)
        vel = torch.from_numpy(vel64).to(dev)
    hist_d = torch.from_numpy(np.ascontiguousarray(hist)).to(dev)
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=w.n_hist, precision=precision,
                 sqrtPnu_init=pi, theta_over_delta_init=ti)
    a = w.a_kick
    K = pm.kick_factor(a, a * 1.01)
    acc = torch.empty_like(vel) if keep_acc else None
    tuned = pm.autotune(pos, vel, a, a_hist, hist_d, reps=1) if autotune else []  # kick factor 0
    if tuning_out is not None:
        tuning_out.extend(tuned)

    def step(out=None):
        if mlp is None:
            pm.nu_prepare(a, a_hist, hist_d)
        pm.deposit(pos)
        if mlp is None:
            pm.nu_response(a, a_hist, hist_d)
        else:
            pm.nu_response_mlp(mlp, a, a_hist, hist_d)
        pm.kick(pos, vel, a, K, acc_out=out)

    for _ in range(warmup):
        step(acc)
    torch.cuda.synchronize()
    pm.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    st = pm.get_timing()
    pm.timing(False)
    pm.check()
    if stages_out is not None:
        stages_out.update({k: v[0] / steps for k, v in st.items() if v[1] > 0})
    ms = e0.elapsed_time(e1) / steps
    pm.close()
    del pos, vel, hist_d
    return ms, st["response"][0] / steps, acc


def _step_form(w, pos64, vel64, steps, warmup):
    """ms per pm_step (kick + P_M store + drift) and per kick alone, FP32 form,
    from the workload's stored history, the drift of each step Delta s to the
    next epoch."""
    import torch
    from paper_1209_0461_gb300 import nupm
    dev = torch.device("cuda")
    a_hist, hist = synth.history(w)
    pi, ti = synth.nu_initial(w)
    pos = torch.from_numpy(synth.to_cell_offset(pos64, w.box, w.ngrid)).to(dev)
    vel = torch.from_numpy(vel64.astype(np.float32)).to(dev)
    hist_d = torch.from_numpy(np.ascontiguousarray(hist)).to(dev)
    n = warmup + steps
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                 a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=w.n_hist + n + 1, precision="fp32",
                 sqrtPnu_init=pi, theta_over_delta_init=ti)
    pm.autotune(pos, vel, w.a_kick, a_hist, hist_d, reps=1)
    pm.history_set(a_hist, hist_d)
    a_steps = w.a_kick * np.exp(0.002 * np.arange(n + 1))
    fac = [(pm.kick_factor(a_steps[j], a_steps[j + 1]), pm.drift_factor(a_steps[j], a_steps[j + 1]))
           for j in range(n)]
    for j in range(warmup):
        pm.step(pos, vel, a_steps[j], *fac[j])
    torch.cuda.synchronize()
    pm.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for j in range(warmup, n):
        pm.step(pos, vel, a_steps[j], *fac[j])
    e1.record()
    torch.cuda.synchronize()
    st = pm.get_timing()
    pm.timing(False)
    pm.check()
    ah, _, _ = pm.history_get()
    ms = e0.elapsed_time(e1) / steps
    pm.close()
    return {"workload": w.name, "ms_per_step": round(ms, 3), "drift_ms": round(st["drift"][0] / steps, 4),
            "kicks_per_s": w.npart / (ms / 1e3), "history_rows_after": int(len(ah))}


def _rms_rel(acc, ref):
    """RMS over particles of |a - a_ref| / RMS |a_ref| (measurement only)."""
    d = (acc.double() - ref.double()).pow(2).sum(0).mean().sqrt()
    return float((d / ref.double().pow(2).sum(0).mean().sqrt()).item())


def run_batched(steps=10, warmup=3):
    """The batched form: 32 boxes (64^3 / 128^3 / 192^3, one particle per cell,
    seeds 0-31, M_nu in {0, 0.06, 0.15, 0.3, 0.6} eV) stepped by one CUDA-graph
    launch -- of the persistent batched passes (one pm_batch per grid size), and
    of the per-box launches on 8 streams after autotuning -- against the same
    32 kicks launched one after another on one stream in FP32 and in FP64;
    force accuracy per box as the RMS of the velocity change against the FP64
    kick."""
    import torch
    from paper_1209_0461_gb300 import batch
    boxes = synth.batched_boxes(32)

    def timed(fn, n, stream):
        # events on the stream the step is issued on (the batch's main stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {"boxes": len(boxes), "particles": int(sum(w.npart for w in boxes))}
    dv = {}
    for name, prec, streams, tune, graph, pers in (("fp64_sequential", "fp64", 1, False, False, False),
                                                   ("fp32_sequential", "fp32", 1, False, False, False),
                                                   ("fp32_graph", "fp32", 8, True, True, False),
                                                   ("fp32_persistent_graph", "fp32", 1, False, True, True)):
        b = batch.Batch(boxes, n_streams=streams, autotune=tune, precision=prec, persistent=pers)
        if graph:
            b.capture()
            step = b.step
            if pers:
                out["persistent_graph_nodes"] = b.graph.nodes()
                out["persistent_launches_per_step"] = b.launches_per_step()
            else:
                out["graph_nodes"] = b.graph.nodes()
                out["tuning"] = {str(k): list(v) for k, v in b.tuning.items()}
        else:
            step = b.eager_step
        b.reset_velocities()
        step()
        b.check()
        torch.cuda.synchronize()
        dv[name] = [(it["vel"] - it["vel0"]).double() for it in b.items]
        for _ in range(warmup):
            step()
        ms = timed(step, steps, b.main)
        b.check()
        out[name] = {"ms_per_step": round(ms, 3), "kicks_per_s": b.npart / (ms / 1e3)}
        b.close()
        torch.cuda.empty_cache()
    for name in ("fp32_sequential", "fp32_graph", "fp32_persistent_graph"):
        errs = [float(((x - r).pow(2).sum(0).mean().sqrt() / r.pow(2).sum(0).mean().sqrt()).item())
                for x, r in zip(dv[name], dv["fp64_sequential"])]
        out[name]["force_rms_rel_vs_fp64_max"] = max(errs)
    out["graph_speedup_vs_fp32_sequential"] = round(out["fp32_sequential"]["ms_per_step"] /
                                                     out["fp32_graph"]["ms_per_step"], 2)
    out["graph_speedup_vs_fp64_sequential"] = round(out["fp64_sequential"]["ms_per_step"] /
                                                     out["fp32_graph"]["ms_per_step"], 2)
    out["persistent_speedup_vs_per_box_graph"] = round(out["fp32_graph"]["ms_per_step"] /
                                                        out["fp32_persistent_graph"]["ms_per_step"], 2)
    return out


def run_forms(steps=3, warmup=1):
    """The FP64 kick against the FP32 (precision) form on the 1024^3 workload,
    and the surrogate form on 512^3 particles / 512^3 grid, each with its force
    accuracy against the plain FP64 GPU kick on the same particles."""
    import torch
    from paper_1209_0461_gb300 import nupm, surrogate
    out = {"batched": run_batched()}
    torch.cuda.empty_cache()
    # precision form vs plain FP64
    w = synth.WORKLOADS["pm1024_p512_fp32"]
    parts = synth.particles(w)
    ms64, r64, acc64 = _kick_form(synth.with_(w, precision="fp64"), parts["pos64"], parts["vel"], "fp64",
                                  steps, warmup)
    ms32, r32, acc32 = _kick_form(w, parts["pos64"], parts["vel"], "fp32", steps, warmup)
    out["fp64_vs_fp32"] = {"workload": w.name, "fp64_ms_per_kick": round(ms64, 3),
                           "fp32_ms_per_kick": round(ms32, 3), "speedup": round(ms64 / ms32, 2),
                           "fp32_force_rms_rel_vs_fp64": _rms_rel(acc32, acc64)}
    # the FP64 path's roofline: max(compulsory HBM bytes / HBM peak, transform
    # flops / measured FP64 FMA rate); two real 3-D transforms of N^3 points a
    # kick (forward delta, inverse potential) at 2.5 N^3 log2 N^3 flops each
    hbm, peak_kind = peaks()
    w64 = synth.with_(w, precision="fp64")
    fma = nupm.measure_fp64_fma()
    M3 = w.ngrid ** 3
    flops = 2 * 2.5 * M3 * math.log2(M3)
    bytes64 = sum(stage_bytes(w64, k, fused_interp=False) for k in
                  ("deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_fwd", "bins", "green", "fft_z_inv", "fft_y_inv",
                   "fft_x_inv", "interp"))
    t_hbm, t_fma = bytes64 / (hbm * 1e9), flops / (fma * 1e12)
    out["fp64_vs_fp32"]["fp64_roofline"] = {
        "bound": "fp64_alu" if t_fma > t_hbm else "hbm", "flops_per_kick": flops, "fp64_fma_tflops": round(fma, 3),
        "bytes_per_kick": bytes64, "hbm_gbs": hbm, "hbm_peak_kind": peak_kind,
        "t_bound_ms": round(max(t_hbm, t_fma) * 1e3, 2), "t_hbm_ms": round(t_hbm * 1e3, 2),
        "t_fma_ms": round(t_fma * 1e3, 2), "frac": round(max(t_hbm, t_fma) * 1e3 / ms64, 4)}
    del acc64, acc32
    torch.cuda.empty_cache()
    # the step loop (Sec. 4.3): pm_step = deposit, response over the context's
    # history, kick, P_M row stored, drift -- against the kick alone
    out["step_loop"] = _step_form(w, parts["pos64"], parts["vel"], steps, warmup)
    del parts
    torch.cuda.empty_cache()
    # the plain FP32 kick at 256^3 / 256^3 (two neutrino masses): throughput and
    # force accuracy against the FP64 GPU kick of the same particles (the FP64
    # oracle comparison of every particle is tests/test_gpu_config2.py)
    out["config2"] = {}
    for name in ("pm256_fp32_m015", "pm256_fp32_m030"):
        w2 = synth.WORKLOADS[name]
        p2 = synth.particles(w2)
        m64, _, a64 = _kick_form(synth.with_(w2, precision="fp64"), p2["pos64"], p2["vel"], "fp64", steps, warmup)
        m32, _, a32 = _kick_form(w2, p2["pos64"], p2["vel"], "fp32", 10, 3)
        out["config2"][name] = {"fp32_ms_per_kick": round(m32, 3), "kicks_per_s": w2.npart / (m32 / 1e3),
                                "fp64_ms_per_kick": round(m64, 3),
                                "fp32_force_rms_rel_vs_fp64_gpu": _rms_rel(a32, a64)}
        del a64, a32, p2
        torch.cuda.empty_cache()
    # the FP64 kick at 32^3 / 32^3 (launch-bound: a few microseconds of work a pass)
    w1 = synth.WORKLOADS["pm32_fp64"]
    p1 = synth.particles(w1)
    m1, r1, _ = _kick_form(w1, p1["pos64"], p1["vel"], "fp64", 50, 5, keep_acc=False, autotune=False)
    out["config1"] = {"pm32_fp64": {"fp64_ms_per_kick": round(m1, 4), "kicks_per_s": w1.npart / (m1 / 1e3),
                                    "response_ms": round(r1, 4)}}
    # contention variant: the same workload with the particles at their a = 1
    # Zel'dovich positions (clustered), reported separately
    wc = synth.with_(w, clustered=True)
    parts = synth.particles(wc)
    msc, _, _ = _kick_form(wc, parts["pos64"], parts["vel"], "fp32", steps, warmup, keep_acc=False,
                           stages_out=(st := {}), tuning_out=(tc := []))
    out["clustered"] = {"workload": w.name + " (Zel'dovich positions at a = 1)", "ms_per_kick": round(msc, 3),
                        "kicks_per_s": w.npart / (msc / 1e3), "tuning": tc,
                        "stages_ms": {k: round(v, 4) for k, v in st.items()}}
    del parts
    torch.cuda.empty_cache()
    # surrogate form
    w = synth.WORKLOADS["pm512_p512_fp32"]
    t0 = time.time()
    X, y, _, _ = surrogate.build_set(64, 64, seed0=0, n_kbins=256, n_hist_max=128)
    Xv, yv, _, fv = surrogate.build_set(8, 16, seed0=5000, n_kbins=256, n_hist_max=128)
    t_gen = time.time() - t0
    mlp = nupm.MLP()
    mlp.set_params(surrogate.init_params(0))
    surrogate.fit_norm(mlp, X, y)
    t0 = time.time()
    hist = surrogate.train(mlp, X, y, epochs=80, batch=4096, lr0=2e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    rel, force = surrogate.errors(mlp, Xv, yv, fv)
    parts = synth.particles(w)
    ms64, _, acc64 = _kick_form(synth.with_(w, precision="fp64"), parts["pos64"], parts["vel"], "fp64",
                                steps, warmup)
    msx, rx, accx = _kick_form(w, parts["pos64"], parts["vel"], "fp32", steps, warmup)
    msm, rm, accm = _kick_form(w, parts["pos64"], parts["vel"], "fp32", steps, warmup, mlp=mlp)
    out["surrogate"] = {
        "workload": w.name, "train_samples": int(X.shape[0]), "gen_s": round(t_gen, 1),
        "train_s": round(t_train, 1), "epochs": len(hist), "final_loss": hist[-1],
        "val_rel_R_median": float(np.median(rel)), "val_rel_R_p99": float(np.percentile(rel, 99)),
        "val_force_bound_max": float(np.max(force)),
        "fp64_exact_ms_per_kick": round(ms64, 3), "fp32_exact_ms_per_kick": round(msx, 3),
        "fp32_surrogate_ms_per_kick": round(msm, 3),
        "response_ms_exact": round(rx, 4), "response_ms_surrogate": round(rm, 4),
        "force_rms_rel_surrogate_vs_fp64": _rms_rel(accm, acc64),
        "force_rms_rel_exact_fp32_vs_fp64": _rms_rel(accx, acc64),
        "force_rms_rel_surrogate_vs_exact_fp32": _rms_rel(accm, accx)}
    mlp.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="pm1024_p512_fp32", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64 / surrogate comparisons")
    ap.add_argument("--no-autotune", action="store_true", help="built-in tile choices instead of pm_autotune")
    ap.add_argument("--tuning", default=None,
                    help="wide_y,wide_z,ctas_per_sm for pm_set_tuning (implies --no-autotune)")
    ap.add_argument("--spectral-gradient", action="store_true",
                    help="gradient as its Fourier multiplier (three force grids) instead of the real-space stencil")
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dtype = "f32" if w.precision == "fp32" else "f64"
    config = {"workload": w.name, "grid": w.ngrid, "particles": w.npart, "box_mpc_h": w.box,
              "m_nu_ev": w.m_nu_total, "n_species": w.n_species, "n_kbins": w.n_kbins,
              "n_hist": w.n_hist, "a": w.a_kick, "positions": "int32 cell + fp32 offset"
              if w.precision == "fp32" else "fp64", "response": "fp64",
              "l2": "inputs larger than L2 (each grid >= 4 GB)", "parallelism": f"replicas x{args.gpus}",
              "gradient": "4-point multiplier -i D(k) in Fourier space" if args.spectral_gradient
              else "4-point stencil on the real potential grid"}
    base = {"metric": "particle-kicks/s incl. neutrino response", "unit": "particle-kicks/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded BBKS Gaussian field, Zel'dovich particles)", "config": config}
    if args.impl == "reference":
        if rank != 0:
            return
        s = oracle_sample(w)
        model, ncpu = host_info()
        oc = OracleCores(w.name)
        for _ in range(args.warmup):
            oc.run()
        rates, walls = [], []
        for _ in range(args.steps):
            v, wall = oc.run()
            rates.append(v)
            walls.append(wall)
        oc.close()
        v = float(np.mean(rates))
        sample = (f"per step one oracle kick on each of {oc.cores} host cores, each a {s.ngrid}^3 grid with "
                  f"{s.npart_side}^3 particles (box {s.box:g} Mpc/h, same cell size, bins and history, "
                  f"its own seed); CPU {model}")
        line = dict(base, impl="reference", value=v, ms_per_step=float(np.mean(walls)) * 1e3,
                    cpu_baseline={"value": v, "unit": "particle-kicks/s", "cores": oc.cores, "kind": "oracle",
                                  "sample": sample, "cpu_model": model, "nproc": ncpu},
                    e2e={"value": v, "unit": "particle-kicks/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0})
        print(json.dumps(line))
        return
    oc = None
    if world == 1 and not args.no_cpu_baseline:
        oc = OracleCores(w.name)          # spawned before any GPU call
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, w, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if oc is not None:
        s = oracle_sample(w)
        model, ncpu = host_info()
        t1, npart = run_oracle_kick(s)          # one core alone
        v_all, wall = oc.run()                  # every core, one kick each
        oc.close()
        cpu = {"value": v_all, "unit": "particle-kicks/s", "cores": oc.cores, "kind": "oracle",
               "sample": f"one oracle kick on each of {oc.cores} host cores ({wall:.1f} s wall), each a "
                         f"{s.ngrid}^3 grid with {s.npart_side}^3 particles (box {s.box:g} Mpc/h, same cell "
                         f"size, bins and history, own seed)",
               "single_core": {"value": npart / t1, "seconds": round(t1, 2)},
               "cpu_model": model, "nproc": ncpu}
    forms = None
    if world == 1 and not args.no_forms and args.workload == "pm1024_p512_fp32":
        forms = run_forms()
    line = dict(base, value=res["value"], ms_per_step=res["ms_per_step"],
                ms_per_step_median=res["ms_per_step_median"], graph=res["graph"], e2e=res["e2e"],
                roofline=res["roofline"], cpu_baseline=cpu, gpu_launches=res["gpu_launches"],
                clocks=res["clocks"], step_model_gb=res["step_alg_gb"], step_hbm_frac=res["step_frac"],
                stages_ms=res["stages"], tuning=res["tuning"], forms=forms)
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
