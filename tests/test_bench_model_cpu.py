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
