"""CPU FP64 oracle of the learned response surrogate.

TEST INFRASTRUCTURE ONLY: imported by the test-suite and by the CPU legs of
``bench.py``; the product path never imports it and shares no code with it.

The surrogate stands in for the linear-response integral (Eq. P-final with
Eq. deltaI-nu) of a kick: per k bin it maps

    x = (ln k_b, ln a, M_nu [eV], Omega_nu, c_0 .. c_7)

to y = ln R_b, R_b = delta_nu / delta_cdm of that bin.  c_j are the Chebyshev
coefficients of the stored total-matter history of the bin, taken relative to
the current CDM amplitude:

    g(u) = ln( P_M^{1/2}(k_b, a'(u)) / P_cdm^{1/2}(k_b, a) ),  u = ln a' in [ln a_i, ln a],

with P_M^{1/2} linear in ln a' between the stored nodes (the same reading of
"interpolating over our tables" as the exact integral), the current node
(ln a, P_cdm^{1/2}) closing the table and the first node held constant back to
a_i.  The network is a 3-layer perceptron of width W:

    h1 = tanh(W1 xh + b1),  h2 = tanh(W2 h1 + b2),  out = w3 . h2 + b3,
    xh = (x - mu) / sigma,  y = y_mu + y_sigma out,

with BF16 weight matrices (W1, W2, w3; FP32 biases), trained on the squared
error of out against (y - y_mu) / y_sigma by Adam.  Nothing here comes from the
paper, which has no learned part: the paper fixes only what the surrogate
replaces.  Each function says what pins it (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import math

import numpy as np

N_CHEB = 8
N_FEATURES = 4 + N_CHEB


# --------------------------------------------------------------------------
# History features
# --------------------------------------------------------------------------
def cheb_nodes(n: int = N_CHEB) -> np.ndarray:
    """t_m = cos(pi (m + 1/2) / n), m = 0..n-1: the Chebyshev points of T_n.

    Pinned by: T_n(t_m) = 0 at every node."""
    m = np.arange(n, dtype=np.float64)
    return np.cos(np.pi * (m + 0.5) / n)


def cheb_coeffs(g_at_nodes: np.ndarray) -> np.ndarray:
    """c_j = (2/n) sum_m g(t_m) T_j(t_m), j = 0..n-1 (discrete orthogonality).

    Then g(t) = c_0 / 2 + sum_{j>=1} c_j T_j(t) for every polynomial g of degree
    < n.  Pinned by: exact recovery of random polynomials of degree 7 built
    with numpy.polynomial.chebyshev."""
    g = np.asarray(g_at_nodes, dtype=np.float64)
    n = g.shape[-1]
    m = np.arange(n, dtype=np.float64)
    j = np.arange(n, dtype=np.float64)[:, None]
    T = np.cos(j * np.pi * (m + 0.5) / n)          # T_j(t_m)
    return (2.0 / n) * g @ T.T


def history_log_ratio(u, a_init: float, a: float, a_hist, sqrtPM_hist_b, sqrtPcdm_b: float):
    """g(u) of one bin at u = ln a' (array): ln of the interpolated history over
    the current CDM amplitude.  Nodes: (ln a_hist[j], sqrtPM_hist_b[j]) and the
    closing node (ln a, sqrtPcdm_b); P_M^{1/2} is linear in ln a' between nodes
    and equal to the first node's value on [ln a_i, ln a_hist[0]].

    Pinned by: the value at every node, linearity between nodes, the constant
    head, and g = 0 without history."""
    u = np.asarray(u, dtype=np.float64)
    un = np.concatenate([np.log(np.asarray(a_hist, dtype=np.float64)), [math.log(a)]])
    hn = np.concatenate([np.asarray(sqrtPM_hist_b, dtype=np.float64), [sqrtPcdm_b]])
    h = np.interp(u, un, hn)                       # constant beyond the first node
    return np.log(h / sqrtPcdm_b)


def features(kb, a: float, m_nu: float, omega_nu: float, a_init: float, a_hist, sqrtPM_hist, sqrtPcdm):
    """Surrogate inputs of every bin: [nk, 12] = (ln k_b, ln a, M_nu, Omega_nu, c_0..c_7).

    sqrtPM_hist: [n_hist, nk]; sqrtPcdm: [nk] (the current measured amplitude).
    The Chebyshev points map to u = ln a_i + (t + 1)/2 (ln a - ln a_i).

    Pinned by: a history with g linear in u gives c_0 = 2 g(mid), c_1 = slope *
    half-width and c_j = 0 beyond; the layout of the first four columns."""
    kb = np.asarray(kb, dtype=np.float64)
    nk = kb.shape[0]
    t = cheb_nodes()
    ui, ua = math.log(a_init), math.log(a)
    u = ui + 0.5 * (t + 1.0) * (ua - ui)
    X = np.zeros((nk, N_FEATURES))
    X[:, 0] = np.log(kb)
    X[:, 1] = math.log(a)
    X[:, 2] = m_nu
    X[:, 3] = omega_nu
    hist = np.asarray(sqrtPM_hist, dtype=np.float64).reshape(len(a_hist), nk)
    for b in range(nk):
        g = history_log_ratio(u, a_init, a, a_hist, hist[:, b], float(sqrtPcdm[b]))
        X[b, 4:] = cheb_coeffs(g)
    return X


# --------------------------------------------------------------------------
# BF16 rounding
# --------------------------------------------------------------------------
def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (8-bit exponent, 7 stored mantissa
    bits), ties to even, returned as FP64.  BF16 is the upper half of an IEEE
    binary32: keep bits 31..16 after adding 0x7FFF + (bit 16).

    Pinned by: exactly representable values unchanged, halfway cases to even,
    relative error <= 2^-8 on random values."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------
def param_sizes(n_in: int, width: int):
    """Flat parameter layout: W1 [width][n_in], b1 [width], W2 [width][width],
    b2 [width], w3 [width], b3 [1]."""
    return [("W1", (width, n_in)), ("b1", (width,)), ("W2", (width, width)), ("b2", (width,)),
            ("w3", (width,)), ("b3", (1,))]


def n_params(n_in: int, width: int) -> int:
    return sum(int(np.prod(s)) for _, s in param_sizes(n_in, width))


def unpack(theta, n_in: int, width: int):
    out, o = {}, 0
    for name, shape in param_sizes(n_in, width):
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(P, n_in: int, width: int) -> np.ndarray:
    return np.concatenate([np.asarray(P[name], dtype=np.float64).ravel() for name, _ in param_sizes(n_in, width)])


def effective(theta, n_in: int, width: int):
    """Parameters as the forward pass uses them: BF16-rounded weight matrices,
    biases as stored (FP32)."""
    P = unpack(theta, n_in, width)
    for name in ("W1", "W2", "w3"):
        P[name] = bf16_round(P[name])
    for name in ("b1", "b2", "b3"):
        P[name] = np.asarray(P[name], dtype=np.float32).astype(np.float64)
    return P


def forward(P, Xh):
    """out[n] of normalised inputs Xh [n, n_in] with parameter dict P (FP64).

    Pinned by: a hand-computed 2-input network; the backward pass's finite
    differences."""
    h1 = np.tanh(Xh @ P["W1"].T + P["b1"])
    h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
    return h2 @ P["w3"] + P["b3"][0], (h1, h2)


def loss_and_grad(P, Xh, Yh):
    """Mean squared error L = (1/n) sum (out - Yh)^2 and dL/dP by the chain rule
    (FP64), for the parameters as given (no rounding inside).

    Pinned by: central finite differences of L in every parameter group."""
    n = Xh.shape[0]
    out, (h1, h2) = forward(P, Xh)
    r = out - Yh
    L = float(np.mean(r * r))
    dout = 2.0 * r / n
    g = {"w3": h2.T @ dout, "b3": np.array([dout.sum()])}
    dz2 = np.outer(dout, P["w3"]) * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ Xh
    g["b1"] = dz1.sum(0)
    return L, g


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) on flat FP64 arrays,
    step t >= 1.  Returns (theta, m, v).

    Pinned by: a hand-computed first step (theta - lr sign(g) for |g| >> eps)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict_lnR(theta, norm, X, n_in: int = N_FEATURES, width: int = 128):
    """ln R of raw features X with the stored normalisation
    norm = (mu [n_in], sigma [n_in], y_mu, y_sigma) and BF16 weights."""
    mu, sig, ymu, ysig = norm
    Xh = (np.asarray(X, dtype=np.float64) - mu) / sig
    out, _ = forward(effective(theta, n_in, width), Xh)
    return ymu + ysig * out
