"""Pins of the surrogate oracle (oracle/mlp_oracle.py) against mathematics it
must reproduce: Chebyshev orthogonality, interpolation at the nodes, BF16
rounding rules, the chain rule (finite differences) and Adam's first step."""
import math

import numpy as np
from numpy.polynomial import chebyshev as C

from oracle import mlp_oracle as M


def test_cheb_nodes_are_roots_of_T8():
    t = M.cheb_nodes()
    assert np.max(np.abs(C.chebval(t, [0] * 8 + [1]))) < 1e-14


def test_cheb_coeffs_recover_polynomials():
    rng = np.random.default_rng(3)
    t = M.cheb_nodes()
    for _ in range(5):
        c = rng.normal(size=8)
        g = C.chebval(t, np.concatenate([[c[0] / 2], c[1:]]))
        assert np.allclose(M.cheb_coeffs(g), c, atol=1e-13)


def test_history_log_ratio_nodes_head_and_linearity():
    a_init, a = 0.02, 0.1
    a_hist = np.array([0.03, 0.05, 0.07])
    h = np.array([2.0, 3.0, 5.0])
    hc = 8.0
    u = np.log(np.concatenate([a_hist, [a]]))
    g = M.history_log_ratio(u, a_init, a, a_hist, h, hc)
    assert np.allclose(g, np.log(np.concatenate([h, [hc]]) / hc), atol=1e-15)
    # constant head back to a_i
    assert abs(M.history_log_ratio(math.log(0.021), a_init, a, a_hist, h, hc) - math.log(2.0 / 8.0)) < 1e-15
    # linear in ln a' between nodes (of P_M^{1/2}, not of its log)
    um = 0.25 * u[1] + 0.75 * u[2]
    assert abs(M.history_log_ratio(um, a_init, a, a_hist, h, hc) - math.log((0.25 * 3 + 0.75 * 5) / 8)) < 1e-14
    # no history: the closing node alone, g = 0
    assert abs(M.history_log_ratio(math.log(0.05), a_init, a, [], [], hc)) < 1e-15


def test_features_of_a_power_law_history():
    # H(u) = h_cur exp(s (u - u_a)) on dense nodes: g is linear in u, so
    # c_0 = 2 g(mid), c_1 = s (u_a - u_i) / 2 and c_j ~ 0 beyond
    a_init, a, s = 0.02, 0.5, 0.8
    nk = 3
    a_hist = np.exp(np.linspace(math.log(a_init), math.log(a), 4001)[:-1])
    hc = np.array([1.0, 2.0, 4.0])
    hist = hc[None, :] * np.exp(s * (np.log(a_hist) - math.log(a)))[:, None]
    X = M.features([0.01, 0.1, 1.0], a, 0.3, 0.0066, a_init, a_hist, hist, hc)
    assert X.shape == (nk, M.N_FEATURES)
    assert np.allclose(X[:, 0], np.log([0.01, 0.1, 1.0])) and np.all(X[:, 1] == math.log(a))
    assert np.all(X[:, 2] == 0.3) and np.all(X[:, 3] == 0.0066)
    ui, ua = math.log(a_init), math.log(a)
    assert np.allclose(X[:, 4], 2 * s * (0.5 * (ui + ua) - ua), atol=1e-6)
    assert np.allclose(X[:, 5], s * (ua - ui) / 2, atol=1e-6)
    assert np.max(np.abs(X[:, 6:])) < 1e-6


def test_bf16_rounding():
    exact = np.array([0.0, 1.0, -2.0, 1.5, 0.0078125, 3.0e38], dtype=np.float32)
    r = M.bf16_round(exact)
    assert np.all(r[:5] == exact[:5].astype(np.float64))
    # halfway cases go to the even mantissa
    assert M.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert M.bf16_round(-(1.0 + 2.0 ** -8)) == -1.0
    x = np.random.default_rng(1).normal(size=10000).astype(np.float32)
    rel = np.abs(M.bf16_round(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8


def test_forward_hand_computed():
    P = {"W1": np.array([[1.0, -1.0], [0.5, 2.0]]), "b1": np.array([0.1, -0.2]),
         "W2": np.array([[1.0, 0.0], [-1.0, 1.0]]), "b2": np.array([0.0, 0.3]),
         "w3": np.array([2.0, -1.0]), "b3": np.array([0.5])}
    x = np.array([[0.3, -0.4]])
    h1 = np.tanh([0.3 + 0.4 + 0.1, 0.15 - 0.8 - 0.2])
    h2 = np.tanh([h1[0], -h1[0] + h1[1] + 0.3])
    out, _ = M.forward(P, x)
    assert abs(out[0] - (2 * h2[0] - h2[1] + 0.5)) < 1e-15


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(5)
    n_in, width, n = 12, 16, 40
    theta = rng.normal(scale=0.4, size=M.n_params(n_in, width))
    X = rng.normal(size=(n, n_in))
    Y = rng.normal(size=n)
    P = M.unpack(theta, n_in, width)
    L, g = M.loss_and_grad(P, X, Y)
    gflat = M.pack(g, n_in, width)
    idx = rng.choice(theta.size, 60, replace=False)
    # every parameter group is represented
    idx = np.concatenate([idx, [0, width * n_in, width * n_in + width + 3, theta.size - width - 1, theta.size - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_and_grad(M.unpack(tp, n_in, width), X, Y)[0] -
              M.loss_and_grad(M.unpack(tm, n_in, width), X, Y)[0]) / (2 * h)
        assert abs(fd - gflat[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_adam_first_step():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t1, m, v = M.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
