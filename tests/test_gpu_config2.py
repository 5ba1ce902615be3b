"""The plain FP32 kick at its own size: 256^3 particles on a 256^3 grid, box
512 Mpc/h, Zel'dovich particles at a = 0.1 from the seeded BBKS field (ICs at
a = 0.02), M_nu = 0.15 and 0.3 eV (three degenerate species), a 64-step
stored history and 128 log-k bins; the response integral in FP64.  Every
output is compared with the FP64 oracle on the same particles: the deposit
bit for bit, R per non-empty bin, and the force of every particle (RMS
relative error, the FP32 path's accuracy bar)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib, force_errors, gpu_kick, make_inputs, oracle_kick  # noqa: E402
from paper_1209_0461_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


@pytest.mark.parametrize("name", ["pm256_fp32_m015", "pm256_fp32_m030"])
def test_fp32_kick_256_against_fp64_oracle(name):
    w = synth.WORKLOADS[name]
    assert (w.ngrid, w.npart, w.n_kbins, w.n_hist, w.precision) == (256, 256 ** 3, 128, 64, "fp32")
    inp = make_inputs(w)
    g = gpu_kick(w, inp)
    r = oracle_kick(w, inp)
    assert np.array_equal(g["F"].astype(np.int64), r.F)
    cnt = g["bins"][0]
    assert np.array_equal(cnt, r.bins["count"])
    ne = r.bins["nonempty"]
    relR = np.abs(g["R"][ne] - r.response["R"][ne]) / np.abs(r.response["R"][ne])
    emax, erms = force_errors(g["acc"], r.acc)
    print(f"{name}: R max rel {relR.max():.2e}, force rms rel {erms:.2e}, max {emax:.2e}")
    assert relR.max() < 1e-5
    assert erms < 2e-4
    dv = g["vel"] - g["vel0"]
    assert np.max(np.abs(dv - g["acc"] * 0.01)) < 1e-5 * np.max(np.abs(dv))
