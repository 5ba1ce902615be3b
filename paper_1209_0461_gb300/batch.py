"""Batched form: many independent boxes stepped by one CUDA-graph launch.

Each box is its own context (grid 64^3, 128^3 or 192^3, its own seed and
neutrino mass).  Two ways to step them:

* persistent: the boxes of each grid size form `split` pm_batches
  (round robin), each kick one persistent kernel per pass over the batch's
  boxes (CTAs take (box, item) work from an atomic counter); every batch runs
  on its own stream, so that different passes (a gather beside a transform)
  share the GPU, and one capture records the few launches of every batch;
* per box: the boxes are spread over a few CUDA streams and one capture
  records every box's response panels, deposit, response and kick (each grid
  size autotuned once with pm_autotune).

Torch supplies device memory, streams and events only.
"""
from __future__ import annotations

import numpy as np

from . import nupm, synth


class Batch:
    def __init__(self, boxes, n_streams: int = 8, autotune: bool = True, precision: str = "fp32",
                 persistent: bool = False, split: int = 2):
        import torch
        self.boxes = list(boxes)
        self.persistent = persistent and precision == "fp32"
        self.main = torch.cuda.Stream()
        self.streams = [torch.cuda.Stream() for _ in range(max(1, n_streams))]
        self.items = []
        self.tuning = {}
        for i, w in enumerate(self.boxes):
            st = self.streams[i % len(self.streams)]
            parts = synth.particles(w)
            a_hist, hist = synth.history(w)
            pi, ti = synth.nu_initial(w)
            with torch.cuda.stream(st):
                if precision == "fp32":
                    pos = torch.from_numpy(synth.to_cell_offset(parts["pos64"], w.box, w.ngrid)).cuda()
                    vel = torch.from_numpy(parts["vel"].astype(np.float32)).cuda()
                else:
                    pos = torch.from_numpy(parts["pos64"]).cuda()
                    vel = torch.from_numpy(parts["vel"]).cuda()
                hist_d = torch.from_numpy(np.ascontiguousarray(hist)).cuda()
            pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                         a_init=w.a_init, n_kbins=w.n_kbins, n_hist_max=max(w.n_hist, 1), precision=precision,
                         sqrtPnu_init=pi, theta_over_delta_init=ti, stream=st)
            a = w.a_kick
            self.items.append(dict(w=w, pm=pm, pos=pos, vel=vel, vel0=vel.clone(), a=a, K=pm.kick_factor(a, a * 1.01),
                                   a_hist=np.ascontiguousarray(a_hist), hist=hist_d, stream=st))
        torch.cuda.synchronize()
        self.groups = []
        if self.persistent:
            # `split` pm_batches per grid size, each on its own stream
            sizes = sorted({it["w"].ngrid for it in self.items})
            for n in sizes:
                its_n = [it for it in self.items if it["w"].ngrid == n]
                for j in range(max(1, min(split, len(its_n)))):
                    its = its_n[j::max(1, min(split, len(its_n)))]
                    st = torch.cuda.Stream()
                    self.groups.append(dict(items=its, stream=st,
                                            batch=nupm.BatchPM([it["pm"] for it in its], st)))
            autotune = False
        if autotune:
            for it in self.items:
                n = it["w"].ngrid
                if n not in self.tuning:
                    self.tuning[n] = it["pm"].autotune(it["pos"], it["vel"], it["a"], it["a_hist"], it["hist"])
                it["pm"].set_tuning(*self.tuning[n])
        self.graph = None

    def _kick(self, it):
        pm = it["pm"]
        pm.nu_prepare(it["a"], it["a_hist"], it["hist"])   # history panels beside the deposit
        pm.deposit(it["pos"])
        pm.nu_response(it["a"], it["a_hist"], it["hist"])
        pm.kick(it["pos"], it["vel"], it["a"], it["K"])

    def _group_kick(self, g):
        its = g["items"]
        g["batch"].kick([it["pos"] for it in its], [it["vel"] for it in its], [it["a"] for it in its],
                        [it["K"] for it in its], [it["a_hist"] for it in its], [it["hist"] for it in its])

    def launches_per_step(self):
        """Kernel launches of one step."""
        if self.persistent:
            return sum(g["batch"].launches() for g in self.groups)
        return None

    def eager_step(self):
        """Every box's kick, launched directly (no graph)."""
        if self.persistent:
            import torch
            fork = torch.cuda.Event()
            fork.record(self.main)
            for g in self.groups:
                g["stream"].wait_event(fork)
                self._group_kick(g)
            for g in self.groups:
                ev = torch.cuda.Event()
                ev.record(g["stream"])
                self.main.wait_event(ev)
            return
        # per box, on the contexts' streams, forked from and joined to the main stream
        import torch
        fork = torch.cuda.Event()
        fork.record(self.main)
        for st in self.streams:
            st.wait_event(fork)
        for it in self.items:
            self._kick(it)
        for st in self.streams:
            ev = torch.cuda.Event()
            ev.record(st)
            self.main.wait_event(ev)

    def capture(self):
        """Record one step of every box into a CUDA graph (after a warm-up step)."""
        import torch
        self.eager_step()
        torch.cuda.synchronize()
        for it in self.items:
            it["pm"].check()

        def body():
            fork = torch.cuda.Event()
            fork.record(self.main)
            if self.persistent:
                for g in self.groups:
                    g["stream"].wait_event(fork)
                    self._group_kick(g)
                for g in self.groups:
                    ev = torch.cuda.Event()
                    ev.record(g["stream"])
                    self.main.wait_event(ev)
                return
            for st in self.streams:
                st.wait_event(fork)
            for it in self.items:
                self._kick(it)
            for st in self.streams:
                ev = torch.cuda.Event()
                ev.record(st)
                self.main.wait_event(ev)

        self.graph = nupm.Graph.capture(self.main, body)
        return self.graph

    def step(self):
        self.graph.launch(self.main)

    def reset_velocities(self):
        import torch
        torch.cuda.synchronize()
        for it in self.items:
            it["vel"].copy_(it["vel0"])
        torch.cuda.synchronize()

    def check(self):
        import torch
        torch.cuda.synchronize()
        for it in self.items:
            it["pm"].check()

    @property
    def npart(self):
        return sum(it["w"].npart for it in self.items)

    def close(self):
        if self.graph is not None:
            self.graph.close()
        for g in self.groups:
            g["batch"].close()
        for it in self.items:
            it["pm"].close()
