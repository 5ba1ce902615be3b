"""Training set, training loop and evaluation of the learned response surrogate.

The paper has no learned part.  The surrogate (pm_mlp_*, see include/nupm.h)
stands in for the response integral of Eq. P-final: the training targets are
outputs of the library's exact integral (pm_nu_response) on seeded scenarios
(``synth.surrogate_group``) whose P_cdm bins are set with pm_set_power; the
features come from pm_response_features; the network trains on the GPU with
pm_mlp_train_step.  Torch only supplies device memory, slicing and the
shuffle of the training rows; numpy holds the host-side bookkeeping.
"""
from __future__ import annotations

import math

import numpy as np

from . import nupm, synth

N_IN = nupm.MLP_FEATURES
WIDTH = nupm.MLP_WIDTH


def init_params(seed: int = 0) -> np.ndarray:
    """Xavier-uniform weight matrices, zero biases, in the flat layout
    W1 [128][12], b1, W2 [128][128], b2, w3 [128], b3."""
    rng = np.random.default_rng(seed)

    def xavier(fan_out, fan_in):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    parts = [xavier(WIDTH, N_IN).ravel(), np.zeros(WIDTH), xavier(WIDTH, WIDTH).ravel(), np.zeros(WIDTH),
             xavier(1, WIDTH).ravel(), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def build_set(n_groups: int, n_scen: int, seed0: int = 0, n_kbins: int = 256, n_hist_max: int = 128):
    """Features X (CUDA float32 [n, 12]) and targets ln R (CUDA float32 [n]) of
    n_groups neutrino masses x n_scen scenarios x n_kbins bins, from the exact
    response.  Also returns per-row (group, scenario) ids and f_nu per row."""
    import torch
    Xs, ys, ids, fnu = [], [], [], []
    ngrid = 32
    for g in range(n_groups):
        w, kb, scen = synth.surrogate_group(seed0 + g, n_scen, n_kbins, n_hist_max)
        pi, ti = synth.nu_initial_at(kb, w)
        pm = nupm.PM(ngrid, 8, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, w.n_species,
                     a_init=w.a_init, n_kbins=n_kbins, n_hist_max=n_hist_max, precision="fp64",
                     sqrtPnu_init=pi, theta_over_delta_init=ti)
        unit = float(ngrid) ** 6 / w.box ** 3        # psum = P count N^6 / L^3 (units of bins())
        ones = np.ones(n_kbins)
        R = torch.empty(n_kbins, dtype=torch.float64, device="cuda")
        for si, s in enumerate(scen):
            pm.set_power(ones, kb, s["sqrtPcdm"] ** 2 * unit)
            hist = torch.from_numpy(np.ascontiguousarray(s["hist"])).cuda()
            pm.nu_response(s["a"], s["a_hist"], hist, ratio=R)
            X = pm.response_features(s["a"], s["a_hist"], hist)
            r = R.cpu().numpy()
            ok = r > 0
            Xs.append(X[torch.from_numpy(ok).cuda()])
            ys.append(np.log(r[ok]).astype(np.float32))
            ids.append(np.full((int(ok.sum()), 2), (g, si)))
            fnu.append(np.full(int(ok.sum()), w.omega_nu / w.omega_m))
        pm.close()
    X = torch.cat(Xs).contiguous()
    y = torch.from_numpy(np.concatenate(ys)).cuda()
    return X, y, np.concatenate(ids), np.concatenate(fnu)


def fit_norm(mlp, X, y):
    """Feature and target normalisation from the training rows."""
    Xh = X.double().cpu().numpy()
    yh = y.double().cpu().numpy()
    mu, sig = Xh.mean(0), Xh.std(0)
    sig[sig < 1e-6] = 1.0
    mlp.set_norm(mu, sig, float(yh.mean()), float(max(yh.std(), 1e-6)))


def train(mlp, X, y, epochs: int = 30, batch: int = 4096, lr0: float = 2e-3, lr_min: float = 2e-5,
          seed: int = 0, log_every: int = 0):
    """Adam with a cosine learning-rate decay over shuffled mini-batches (one
    reshuffle per epoch).  Returns the per-epoch mean training loss."""
    import torch
    n = int(X.shape[0])
    steps_per_epoch = max(n // batch, 1)
    total = epochs * steps_per_epoch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    loss = torch.zeros(steps_per_epoch, dtype=torch.float32, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        Xs, ys = X[perm].contiguous(), y[perm].contiguous()
        for i in range(steps_per_epoch):
            lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / total))
            sl = slice(i * batch, min((i + 1) * batch, n))
            mlp.train_step(Xs[sl], ys[sl], lr, loss[i:i + 1])
            step += 1
        hist.append(float(loss.mean().item()))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.3e}")
    return hist


def errors(mlp, X, y, f_nu):
    """Per-row |R_mlp - R| / R and f_nu |R_mlp - R| / (1 - f_nu + f_nu R): the
    relative error of R and the relative error it puts on delta_M (and so on
    the force) of that bin."""
    pred = mlp.forward(X).double().cpu().numpy()
    R = np.exp(y.double().cpu().numpy())
    Rm = np.exp(pred)
    rel = np.abs(Rm - R) / R
    force = f_nu * np.abs(Rm - R) / (1.0 - f_nu + f_nu * R)
    return rel, force
