"""The benchmark's algorithmic-byte model (the roofline numerator) on the
1024^3 / 512^3 FP32 workload, checked against the pass-by-pass sums written
out here from the layout: each pass reads its inputs and writes its outputs
once at stored precision."""
import bench
from paper_1209_0461_gb300 import synth

W = synth.WORKLOADS["pm1024_p512_fp32"]
N, NP = 1024, 512 ** 3
CPLX = 8 * N * N * (N // 2)          # one packed complex field, bytes
REAL = 4 * N ** 3                    # one real field, bytes


def test_real_space_gradient_pass_model():
    b = {k: bench.stage_bytes(W, k, False, False) for k in
         ("deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_fwd", "bins", "fft_z_inv", "fft_y_inv", "fft_x_inv", "interp")}
    assert b["deposit"] == 32 * NP                     # positions in, 8-byte records out
    assert b["fft_x_fwd"] == 8 * NP + CPLX             # records in, spectrum out
    assert b["fft_y_fwd"] == b["fft_z_fwd"] == 2 * CPLX
    assert b["bins"] == CPLX
    assert b["fft_z_inv"] == b["fft_y_inv"] == 2 * CPLX  # one field: the potential
    assert b["fft_x_inv"] == CPLX + REAL
    assert b["interp"] == 24 * NP + REAL + 24 * NP      # positions, the potential once, velocities r+w
    total = sum(b.values()) + 3 * 8 * N * N             # + the packed column's Green kernel
    assert abs(total / 1e9 - 67.7) < 0.1


def test_spectral_gradient_carries_three_fields():
    z = bench.stage_bytes(W, "fft_z_inv", False, True)
    y = bench.stage_bytes(W, "fft_y_inv", False, True)
    x = bench.stage_bytes(W, "fft_x_inv", False, True)
    assert z == 3 * CPLX and y == 5 * CPLX and x == 3 * (CPLX + REAL)


def test_bin_sums_in_the_z_pass():
    # FP32, wide_z = 2 (TMA-staged z passes), at most 256 bins, a power-of-two
    # grid of 256 or more: the bins stage reads the packed x2 = 0 column only
    assert bench.bins_in_z(W, [0, 2, 4, 0])
    assert not bench.bins_in_z(W, [0, 1, 4, 0])
    assert not bench.bins_in_z(W, None)
    assert not bench.bins_in_z(synth.with_(W, precision="fp64"), [0, 2, 4, 0])
    assert not bench.bins_in_z(synth.with_(W, n_kbins=512), [0, 2, 4, 0])
    assert not bench.bins_in_z(synth.with_(W, ngrid=192), [0, 2, 4, 0])
    assert bench.stage_bytes(W, "bins", False, False, True) == 8 * N * N
    assert bench.stage_bytes(W, "fft_z_fwd", False, False, True) == 2 * CPLX
    total = sum(bench.stage_bytes(W, k, False, False, True) for k in
                ("deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_fwd", "bins", "fft_z_inv", "fft_y_inv",
                 "fft_x_inv", "interp")) + 3 * 8 * N * N
    assert abs(total / 1e9 - 63.4) < 0.1
