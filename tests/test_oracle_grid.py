"""Pins of the oracle's grid steps: fixed-point CIC deposit, density contrast,
forward DFT, power-spectrum bins, Green/gradient, inverse DFT, interpolation.
Each test checks against brute force, a closed form or a hand computation."""
import math

import numpy as np
import pytest

from oracle import pm_oracle as O


def _brute_deposit(c, w, n):
    F = np.zeros((n, n, n), dtype=object)
    for p in range(c.shape[1]):
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    wx = int(w[0, p]) if dx else 65536 - int(w[0, p])
                    wy = int(w[1, p]) if dy else 65536 - int(w[1, p])
                    wz = int(w[2, p]) if dz else 65536 - int(w[2, p])
                    F[(c[2, p] + dz) % n, (c[1, p] + dy) % n, (c[0, p] + dx) % n] += wx * wy * wz
    return F.astype(np.int64)


def test_single_particle_hand_computed():
    # one particle at grid coordinates (1.25, 2.5, 3.75) on a 4^3 grid, L = 4
    pos = np.array([[1.25], [2.5], [3.75]])
    c, w = O.quantise_positions_f64(pos, 4.0, 4)
    assert c[:, 0].tolist() == [1, 2, 3]
    assert w[:, 0].tolist() == [16384, 32768, 49152]
    F = O.cic_deposit(c, w, 4)
    # z = 3 -> (1 - 0.75), z = 0 (wrapped) -> 0.75; y = 2, 3 -> 0.5 each;
    # x = 1 -> 0.75, x = 2 -> 0.25
    assert F[3, 2, 1] == 49152 * 32768 * 16384
    assert F[0, 3, 2] == 16384 * 32768 * 49152
    assert F[0, 2, 1] == 49152 * 32768 * 49152
    assert int(F.sum()) == 2 ** 48
    assert np.count_nonzero(F) == 8


def test_mass_conservation_and_brute_force():
    rng = np.random.default_rng(1)
    n = 8
    pos = rng.uniform(-20.0, 40.0, size=(3, 300))   # outside the box: wraps
    c, w = O.quantise_positions_f64(pos, 16.0, n)
    F = O.cic_deposit(c, w, n)
    assert int(F.sum()) == 300 * 2 ** 48
    assert np.array_equal(F, _brute_deposit(c, w, n))
    assert np.all((c >= 0) & (c < n)) and np.all((w >= 0) & (w < 65536))


def test_cell_offset_form_and_range_check():
    cell = np.array([[7], [-1], [8]], dtype=np.int32)
    off = np.array([[0.5], [0.0], [0.999999]], dtype=np.float32)
    c, w = O.quantise_positions_cell(cell, off, 8)
    assert c[:, 0].tolist() == [7, 7, 0]
    assert w[:, 0].tolist() == [32768, 0, int(math.floor(np.float64(np.float32(0.999999)) * 65536))]
    with pytest.raises(ValueError):
        O.quantise_positions_cell(cell, np.array([[1.0], [0.0], [0.0]], dtype=np.float32), 8)
    with pytest.raises(ValueError):
        O.quantise_positions_cell(cell, np.array([[-0.1], [0.0], [0.0]], dtype=np.float32), 8)


def test_density_contrast_mean_zero():
    rng = np.random.default_rng(2)
    pos = rng.uniform(0, 10.0, size=(3, 512))
    c, w = O.quantise_positions_f64(pos, 10.0, 8)
    d = O.density_contrast(O.cic_deposit(c, w, 8), 512)
    assert abs(d.mean()) < 1e-14


def test_forward_fft_brute_dft():
    rng = np.random.default_rng(3)
    n = 8
    x = rng.standard_normal((n, n, n))
    j = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(j, j) / n)
    ref = np.einsum("az,by,cx,zyx->abc", W, W, W[: n // 2 + 1], x)
    assert np.max(np.abs(O.forward_fft(x) - ref)) < 1e-11
    # Parseval with the Hermitian weights of the half spectrum
    spec = O.forward_fft(x)
    wgt = np.full(n // 2 + 1, 2.0)
    wgt[0] = wgt[-1] = 1.0
    assert abs((wgt * np.abs(spec) ** 2).sum() / n ** 3 - (x ** 2).sum()) < 1e-9


def test_bin_counts_match_lattice_enumeration():
    for n, nk, box in ((8, 6, 100.0), (16, 12, 50.0)):
        T = O.bin_thresholds(n, nk)
        assert T[0] == 1 and T[-1] > 3 * (n // 2) ** 2
        assert np.all(np.diff(T) >= 0)
        b = O.bin_power(np.ones((n, n, n // 2 + 1), dtype=complex), box, nk)
        cnt = np.zeros(nk)
        ksum = np.zeros(nk)
        f = np.fft.fftfreq(n, 1.0 / n)
        for iz in f:
            for iy in f:
                for ix in f:            # full spectrum: every mode counted once
                    n2 = int(iz * iz + iy * iy + ix * ix)
                    if n2 == 0:
                        continue
                    kb = max(i for i in range(nk) if T[i] <= n2)
                    cnt[kb] += 1
                    ksum[kb] += 2 * math.pi / box * math.sqrt(n2)
        assert np.array_equal(b["count"], cnt)
        assert np.allclose(b["ksum"], ksum, rtol=1e-13, atol=0)
        assert b["count"].sum() == n ** 3 - 1


def test_bin_edges_geometry():
    # edges e_b = kmin (kmax/kmin)^(b/nk): T_b = ceil((e_b L / 2pi)^2)
    n, nk = 64, 20
    r = math.sqrt(3) * n / 2 * (1 + 1e-12)
    T = O.bin_thresholds(n, nk)
    for b in range(nk + 1):
        e2 = r ** (2 * b / nk)
        assert T[b] - 1 < e2 <= T[b]


def test_plane_wave_single_bin():
    n, box, nk, A = 16, 80.0, 10, 0.3
    x = np.arange(n)
    delta = A * np.cos(2 * np.pi * 3 * x / n)[None, None, :] * np.ones((n, n, 1))
    b = O.bin_power(O.forward_fft(delta), box, nk)
    T = b["T"]
    kb = max(i for i in range(nk) if T[i] <= 9)
    nz = np.nonzero(b["psum"] > 1e-12)[0]
    assert nz.tolist() == [kb]
    # |delta_k| = A N^3 / 2 on (kx = 3), weight 2 -> P = A^2 L^3 / (2 count)
    assert abs(b["P"][kb] - A * A * box ** 3 / (2 * b["count"][kb])) < 1e-12 * b["P"][kb]


def test_cosine_mode_acceleration_closed_form():
    # delta = A cos(k0 . x): phi = -1.5 Om A cos / (a k0^2) (Eq. Poisson).  The
    # 4-point difference of a sampled sine of wavenumber k is exactly
    # [8 sin(k D) - sin(2 k D)] / (6 D) times the cosine, so
    # acc_c = -1.5 Om A g_c sin(k0.x) / (a k0^2), g_c that factor per axis.
    n, box, a, A = 16, 64.0, 0.25, 1e-2
    cos = O.Cosmo(omega_cdm=0.3, omega_nu=0.0, h=0.7)
    kf = 2 * np.pi / box
    D = box / n
    for m in ((2, 0, 0), (1, 2, 0), (1, 1, 3), (8, 0, 0)):
        g = np.arange(n) * box / n
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        kvec = np.array(m) * kf
        phase = kvec[0] * X + kvec[1] * Y + kvec[2] * Z
        delta = A * np.cos(phase)
        spec = O.forward_fft(delta)
        nk = 8
        accs = O.green_gradient(spec, box, a, cos, np.ones(nk), np.zeros(nk), np.zeros(nk, bool))
        k2 = (kvec ** 2).sum()
        for comp in range(3):
            got = O.inverse_fft(accs[comp], n)
            gc = (8 * np.sin(kvec[comp] * D) - np.sin(2 * kvec[comp] * D)) / (6 * D)
            ref = -1.5 * 0.3 * A * gc * np.sin(phase) / (a * k2)
            assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_gradient_operator_is_four_point_stencil():
    # Applying the multiplier to a random periodic field equals the real-space
    # stencil [8 (f+1 - f-1) - (f+2 - f-2)] / (12 D) along each axis.
    n, box = 8, 24.0
    rng = np.random.default_rng(9)
    f = rng.standard_normal((n, n, n))
    spec = O.forward_fft(f)
    iz, iy, ix = O.mode_indices(n)
    D = box / n
    for comp, axis in ((ix, 2), (iy, 1), (iz, 0)):
        got = O.inverse_fft(1j * O.gradient_operator(comp, n, box) * spec, n)
        ref = (8 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))
               - (np.roll(f, -2, axis) - np.roll(f, 2, axis))) / (12 * D)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_neutrino_factor_in_green():
    # delta_M = delta_cdm [(1 - f) + f R]: with R == const the force scales by
    # (1 - f) + f R exactly.
    n, box, a = 8, 40.0, 0.5
    rng = np.random.default_rng(5)
    spec = O.forward_fft(rng.standard_normal((n, n, n)))
    c0 = O.Cosmo(0.3, 0.0, 0.7)
    c1 = O.Cosmo(0.27, 0.03, 0.7, (0.1,))
    kb = np.array([0.1, 0.5, 1.0])
    R = np.array([0.4, 0.4, 0.4])
    a0 = O.green_gradient(spec, box, a, c0, kb, R, np.ones(3, bool))
    a1 = O.green_gradient(spec, box, a, c1, kb, R, np.ones(3, bool))
    fac = (1 - 0.1) + 0.1 * 0.4
    for q0, q1 in zip(a0, a1):
        assert np.allclose(q1, q0 * fac, rtol=1e-14, atol=1e-300)


def test_ratio_interpolation_linear_in_lnk():
    kb = np.array([0.1, 0.0, 0.4, 1.6])
    R = np.array([1.0, 9.0, 0.5, 0.25])
    ne = np.array([True, False, True, True])
    k = np.array([0.05, 0.1, 0.2, 0.4, 0.8, 3.0])
    got = O.ratio_per_mode(k, kb, R, ne)
    # between 0.1 and 0.4, ln-spaced: 0.2 is the log-midpoint
    assert np.allclose(got, [1.0, 1.0, 0.75, 0.5, 0.375, 0.25], rtol=1e-14)


def test_interpolation_exact_for_linear_field():
    n = 16
    g = np.zeros((n, n, n))
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    g[:] = 0.5 + 0.25 * ix - 0.125 * iy + 2.0 * iz
    rng = np.random.default_rng(6)
    u = rng.uniform(1.0, n - 2.0, size=(3, 200))
    c, w = O.quantise_positions_f64(u, float(n), n)
    got = O.cic_interpolate(g, c, w)
    uq = c + w / 65536.0
    ref = 0.5 + 0.25 * uq[0] - 0.125 * uq[1] + 2.0 * uq[2]
    assert np.max(np.abs(got - ref)) < 1e-12


def _ewald_grad_G(r, L, alpha=None, nreal=3, nk=8):
    """grad of the periodic Green's function G with lap G = delta_D - 1/L^3
    (Ewald summation), at separation vectors r [3, m]."""
    alpha = 2.0 / L if alpha is None else alpha
    from scipy.special import erfc
    out = np.zeros_like(r)
    rng = range(-nreal, nreal + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                d = r - L * np.array([i, j, k])[:, None]
                s = np.sqrt((d * d).sum(0))
                fac = (erfc(alpha * s) + 2 * alpha * s / np.sqrt(np.pi) * np.exp(-alpha ** 2 * s ** 2))
                out += d / (4 * np.pi * s ** 3) * fac
    kf = 2 * np.pi / L
    rngk = range(-nk, nk + 1)
    for i in rngk:
        for j in rngk:
            for k in rngk:
                if i == j == k == 0:
                    continue
                kv = kf * np.array([i, j, k], dtype=float)
                k2 = (kv * kv).sum()
                out += (kv[:, None] / k2) * np.exp(-k2 / (4 * alpha ** 2)) * np.sin(kv @ r) / L ** 3
    return out


def test_point_mass_against_ewald():
    # One particle: delta = L^3 delta_D - 1, phi solves lap phi = 1.5 Om delta / a,
    # so acc = -1.5 Om L^3 / a grad G_periodic (Ewald).  The PM force (CIC,
    # 4-point gradient, no deconvolution) follows it to ~1% in the median at
    # 4 cells <= r < L/4, with a few-% spread from the mesh anisotropy.
    n, L, a = 64, 64.0, 1.0
    om = 0.3
    cos = O.Cosmo(om, 0.0, 0.7)
    rng = np.random.default_rng(7)
    for x0 in (np.array([[32.0], [32.0], [32.0]]), np.array([[32.3], [31.6], [32.77]])):
        c0, w0 = O.quantise_positions_f64(x0, L, n)
        F = O.cic_deposit(c0, w0, n)
        spec = O.forward_fft(O.density_contrast(F, 1))
        nk = 8
        accs = O.green_gradient(spec, L, a, cos, np.ones(nk), np.zeros(nk), np.zeros(nk, bool))
        fields = [O.inverse_fft(q, n) for q in accs]
        dirs = rng.standard_normal((3, 240))
        dirs /= np.sqrt((dirs ** 2).sum(0))
        radii = rng.uniform(4.0, 16.0, 240)
        pts = x0 + dirs * radii
        c, w = O.quantise_positions_f64(pts, L, n)
        acc = np.stack([O.cic_interpolate(fd, c, w) for fd in fields])
        ref = -1.5 * om * L ** 3 / a * _ewald_grad_G(pts - x0, L)
        err = np.sqrt(((acc - ref) ** 2).sum(0)) / np.sqrt((ref ** 2).sum(0))
        near = radii < 6
        assert np.median(err[near]) < 0.015
        assert np.median(err[~near]) < 0.005
        assert np.max(err) < 0.08
        # attractive: acceleration points back to the mass
        assert np.all((acc * (pts - x0)).sum(0) < 0)


def _random_particles(n, npart, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, n, size=(3, npart)).astype(np.int64)
    w = rng.integers(0, 65536, size=(3, npart)).astype(np.int64)
    return c, w


def test_deposit_at_sampled_cells_equals_brute_force():
    n = 8
    c, w = _random_particles(n, 300, 5)
    c[:, :4] = [[0, n - 1, 0, n - 1], [n - 1, 0, n - 1, 0], [n - 1, n - 1, 0, 0]]   # wrap across every face
    F = _brute_deposit(c, w, n)
    rng = np.random.default_rng(6)
    cells = np.concatenate([[0, n ** 3 - 1, (n - 1) * n * n, n - 1], rng.integers(0, n ** 3, 40)])
    got = O.cic_deposit_cells(c, w, n, cells)
    assert np.array_equal(got, F.reshape(-1)[cells])


def test_density_modes_equal_brute_dft_of_deposit():
    n, npart = 8, 200
    c, w = _random_particles(n, npart, 7)
    F = _brute_deposit(c, w, n).astype(np.float64)
    delta = F * (n ** 3 / (npart * 2.0 ** 48)) - 1.0
    x = np.arange(n)
    modes = [(0, 0, 0), (0, 0, 1), (1, -2, 0), (-3, 2, 4), (-4, -4, 4), (2, 3, 1), (0, -1, 0), (3, 0, 2)]
    kz, ky, kx = (np.array(v) for v in zip(*modes))
    got = O.density_modes(c, w, n, npart, kz, ky, kx, chunk=64)
    for i, (a, b, d) in enumerate(modes):
        ph = np.exp(-2j * math.pi * (a * x[:, None, None] + b * x[None, :, None] + d * x[None, None, :]) / n)
        ref = (delta * ph).sum()
        assert abs(got[i] - ref) < 1e-12 * (1 + abs(ref)), (modes[i], got[i], ref)
    # and against the oracle's own FFT route
    spec = O.forward_fft(O.density_contrast(O.cic_deposit(c, w, n), npart))
    assert np.allclose(got, spec[kz % n, ky % n, kx], rtol=1e-12, atol=1e-10)


def test_bin_power_over_complete_bins_equals_full_bins():
    n, box, nk = 16, 100.0, 12
    rng = np.random.default_rng(8)
    delta = rng.normal(size=(n, n, n))
    spec = O.forward_fft(delta)
    full = O.bin_power(spec, box, nk)
    T = full["T"]
    lim = 13
    iz, iy, ix = O.mode_indices(n)
    n2 = iz * iz + iy * iy + ix * ix
    sel = np.nonzero((n2 < lim) & (n2 > 0))
    part = O.bin_power_modes(spec[sel], iz[sel[0], 0, 0], iy[0, sel[1], 0], ix[0, 0, sel[2]], n, box, nk)
    done = T[1:] <= lim                     # bins all of whose modes have n^2 < lim
    assert done.sum() >= 3
    for key in ("count", "ksum", "psum", "k", "P"):
        assert np.allclose(part[key][done], full[key][done], rtol=1e-13, atol=0), key
    # the potential at a mode subset equals the full spectrum's values there
    cos = O.Cosmo(0.25, 0.05, 0.7, (0.1, 0.1, 0.1), 0.02)
    R = np.linspace(0.2, 0.9, nk)
    phi = O.potential_spectrum(spec, box, 0.1, cos, full["k"], R, full["nonempty"])
    phis = O.potential_spectrum(spec[sel], box, 0.1, cos, full["k"], R, full["nonempty"],
                                modes=(iz[sel[0], 0, 0], iy[0, sel[1], 0], ix[0, 0, sel[2]]), ngrid=n)
    assert np.array_equal(phis, phi[sel])


def _mean_window(n, offsets, weights, axes):
    """Average over particle offsets of the single-particle CIC deposit's DFT
    (oracle deposit + forward FFT, unit mass) times e^{+2 pi i k.x / N}: the
    assignment window W(k) at every half-spectrum mode.  offsets [P, 3] in cell
    units, exact multiples of 2^-16; only the axes listed move."""
    iz, iy, ix = O.mode_indices(n)
    acc = np.zeros((n, n, n // 2 + 1), dtype=complex)
    base = np.array([3, 5, 2])
    for o, wt in zip(offsets, weights):
        u = base + o
        c = np.floor(u).astype(np.int64)[:, None]
        w = np.round((u - np.floor(u)) * 65536).astype(np.int64)[:, None]
        F = O.cic_deposit(c, w, n).astype(np.float64) / O.MASS_ONE
        spec = O.forward_fft(F)
        ph = np.exp(2j * np.pi * (ix * u[0] + iy * u[1] + iz * u[2]) / n)
        acc += wt * spec * ph
    return acc


def test_cic_window_and_its_deconvolution():
    # The CIC assignment window: averaged over a uniform sub-cell offset o, the
    # DFT of one particle's deposit times e^{+2 pi i n x / N} is, per axis,
    #   2 int_0^1 (1 - o) cos(theta o) do = sinc^2(theta / 2),  theta = 2 pi n / N.
    # The deconvolution of potential_spectrum divides by the square of this
    # window (assignment and interpolation): prod sinc^4(pi n_i / N).
    n = 8
    # 1-D: the x offset on the midpoint rule of 1024 exact points
    J = 1024
    o = (np.arange(J) + 0.5) / J
    offs = np.stack([o, np.zeros(J), np.zeros(J)], axis=1)
    W1 = _mean_window(n, offs, np.full(J, 1.0 / J), (0,))
    ix = np.arange(n // 2 + 1)
    t = np.pi * ix / n
    sinc2 = np.where(ix == 0, 1.0, (np.sin(t) / np.where(ix == 0, 1.0, t)) ** 2)
    assert np.allclose(W1, np.broadcast_to(sinc2, W1.shape), atol=2e-6, rtol=0)
    # 3-D: 8-point Gauss-Legendre in each axis (offsets rounded to 2^-16)
    g, gw = np.polynomial.legendre.leggauss(8)
    g = np.round((g + 1) / 2 * 65536) / 65536
    gw = gw / 2
    oz, oy, ox = np.meshgrid(g, g, g, indexing="ij")
    wz, wy, wx = np.meshgrid(gw, gw, gw, indexing="ij")
    offs3 = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1)
    W3 = _mean_window(n, offs3, (wx * wy * wz).ravel(), (0, 1, 2))
    assert np.max(np.abs(W3.imag)) < 1e-4
    # the oracle's deconvolution factor of the Green function is 1 / W^2
    cos = O.Cosmo(0.3, 0.0, 0.7, (), 0.02)
    rng = np.random.default_rng(3)
    spec = rng.normal(size=W3.shape) + 1j * rng.normal(size=W3.shape)
    kb, R, ne = np.ones(4), np.zeros(4), np.zeros(4, bool)
    plain = O.potential_spectrum(spec, 100.0, 0.5, cos, kb, R, ne, deconvolve=False)
    dec = O.potential_spectrum(spec, 100.0, 0.5, cos, kb, R, ne, deconvolve=True)
    sel = plain != 0
    ratio = (dec[sel] / plain[sel]).real
    assert np.allclose(ratio * W3.real[sel] ** 2, 1.0, rtol=3e-4, atol=0)
