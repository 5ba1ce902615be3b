"""The allocation-free P(k) entry point (pm_bin_power_static) against the
context's own bins (pm_get_bins) on the same spectrum, two calls in a row,
and against the oracle's bin sums of that spectrum; at the 256-bin limit on a
128^3 grid (every CTA gets rows, the shared accumulators are used to the end)
and on a small grid right after a large one (no stale partial sums leak
through the shared scratch array).

pm_bin_power_static exists for callers that cannot allocate device memory
(all of it reserved by their own pool at start-up, or no allocation allowed
inside the time-step loop); its scratch is a fixed device array in the
library.  This file is collected last so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _context_spectrum(prec, n, nk):
    """The context's bins and its forward spectrum (rfftn layout, on the device)
    for seeded particles on an n^3 grid."""
    from paper_1209_0461_gb300 import nupm, synth
    w = synth.Workload(f"noalloc{n}", n, min(n, 64), 4.0 * n, 0.3, 3, 2, nk, prec)
    parts = synth.particles(w)
    dev = torch.device("cuda")
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, 3,
                 n_kbins=nk, precision=prec)
    if prec == "fp64":
        pos = torch.from_numpy(parts["pos64"]).to(dev).contiguous()
    else:
        pos = torch.from_numpy(synth.to_cell_offset(parts["pos64"], w.box, w.ngrid)).to(dev).contiguous()
    pm.deposit(pos)
    bins = pm.bins()
    spec = pm.field(nupm.FIELD_DELTA_K)
    pm.close()
    return w, bins, spec


def _static(spec, n, box, nk):
    from paper_1209_0461_gb300 import nupm
    outs = [torch.full((nk,), float("nan"), dtype=torch.float64, device=spec.device) for _ in range(3)]
    nupm.bin_power_static(spec, n, box, nk, *outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("prec,n,nk", [("fp64", 128, 256), ("fp32", 128, 256)])
def test_static_bins_at_the_bin_limit_then_a_small_grid(prec, n, nk):
    from oracle import pm_oracle as O
    from paper_1209_0461_gb300 import build as b
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    b.build()
    w, (cnt, ks, ps), spec = _context_spectrum(prec, n, nk)
    c2, k2, p2 = _static(spec, n, w.box, nk)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.array_equal(c2, cnt)
    assert np.allclose(k2, ks, rtol=1e-13, atol=0)
    assert np.allclose(p2, ps, rtol=tol, atol=1e-300)
    # the oracle's bins of the same spectrum
    ref = O.bin_power(spec.cpu().numpy().astype(np.complex128), w.box, nk)
    assert np.array_equal(c2, ref["count"])
    ne = ref["count"] > 0
    assert ne.sum() == 187 and ne[-1]      # the last of the 256 bins holds modes
    assert np.allclose(k2[ne], ref["ksum"][ne], rtol=1e-12, atol=0)
    assert np.allclose(p2[ne], ref["psum"][ne], rtol=1e-10, atol=0)
    # straight after, a 16^3 grid with 8 bins on the same scratch array
    w16, (c16, k16, p16), s16 = _context_spectrum(prec, 16, 8)
    d16 = _static(s16, 16, w16.box, 8)
    assert np.array_equal(d16[0], c16)
    assert np.allclose(d16[1], k16, rtol=1e-13, atol=0)
    assert np.allclose(d16[2], p16, rtol=tol, atol=1e-300)


@pytest.mark.parametrize("prec,n,nk", [("fp64", 32, 32), ("fp32", 64, 48)])
def test_static_bins_match_context_bins(prec, n, nk):
    from paper_1209_0461_gb300 import build as b
    from paper_1209_0461_gb300 import nupm, synth
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    b.build()
    w = synth.Workload(f"noalloc{n}", n, n, 4.0 * n, 0.3, 3, 2, nk, prec)
    parts = synth.particles(w)
    dev = torch.device("cuda")
    pm = nupm.PM(w.ngrid, w.npart, w.box, w.omega_cdm, w.omega_nu, w.h, w.m_nu_total, 3,
                 n_kbins=nk, precision=prec)   # deposit path as in production (fused)
    if prec == "fp64":
        pos = torch.from_numpy(parts["pos64"]).to(dev).contiguous()
    else:
        pos = torch.from_numpy(synth.to_cell_offset(parts["pos64"], w.box, w.ngrid)).to(dev).contiguous()
    pm.deposit(pos)
    cnt, ks, ps = pm.bins()
    spec = pm.field(nupm.FIELD_DELTA_K)
    tol = 1e-10 if prec == "fp64" else 2e-5
    for call in range(2):
        outs = [torch.full((nk,), float("nan"), dtype=torch.float64, device=dev) for _ in range(3)]
        nupm.bin_power_static(spec, n, w.box, nk, *outs)
        torch.cuda.synchronize()
        c2, k2, p2 = (o.cpu().numpy() for o in outs)
        assert np.array_equal(c2, cnt), call
        assert np.allclose(k2, ks, rtol=1e-13, atol=0), call
        assert np.allclose(p2, ps, rtol=tol, atol=1e-300), call
    pm.close()


def test_static_bins_rejects_too_many_bins():
    from paper_1209_0461_gb300 import nupm
    spec = torch.zeros((16, 16, 9), dtype=torch.complex128, device="cuda")
    with pytest.raises(nupm.PMError) as e:
        nupm.bin_power_static(spec, 16, 32.0, 257)
    assert e.value.code == -2
