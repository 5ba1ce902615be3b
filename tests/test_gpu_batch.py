"""GPU tests of the batched form: boxes of 64^3, 128^3 and 192^3 (mixed radix)
stepped by one CUDA-graph launch give the same velocities, bit for bit, as the
same kicks launched directly; the autotuner's choices do not change results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib  # noqa: E402
from paper_1209_0461_gb300 import batch, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


def _dv(b):
    torch.cuda.synchronize()
    return [(it["vel"] - it["vel0"]).cpu().numpy() for it in b.items]


def test_graph_step_equals_direct_launches():
    boxes = synth.batched_boxes(6, n_hist=8, n_kbins=32)
    b = batch.Batch(boxes, n_streams=3, autotune=True)
    for n, t in b.tuning.items():
        assert t[0] in (0, 1) and t[1] in (0, 1) and t[2] in (4, 8, 16, 32) and t[3] in (0, 1), (n, t)
    b.eager_step()
    b.check()
    ref = _dv(b)
    assert all(np.all(np.isfinite(d)) and np.any(d != 0) for d in ref)
    b.reset_velocities()
    g = b.capture()
    assert g.nodes() >= 6 * 10
    b.reset_velocities()
    b.step()
    b.check()
    got = _dv(b)
    for d0, d1 in zip(ref, got):
        assert np.array_equal(d0, d1)
    # a second launch kicks again from the updated velocities: twice the change
    b.step()
    b.check()
    two = _dv(b)
    for d0, d2 in zip(ref, two):
        assert np.allclose(d2, 2 * d0, rtol=1e-5, atol=1e-6 * np.abs(d0).max())
    b.close()


def test_tuning_does_not_change_results():
    boxes = synth.batched_boxes(3, n_hist=4, n_kbins=24)
    out = []
    for tune in [(0, 0, 4), (1, 1, 32)]:
        b = batch.Batch(boxes, n_streams=1, autotune=False)
        for it in b.items:
            it["pm"].set_tuning(*tune)
        b.eager_step()
        b.check()
        out.append(_dv(b))
        b.close()
    for d0, d1 in zip(*out):
        assert np.array_equal(d0, d1)


def test_persistent_batch_matches_direct_kicks_and_graphs_to_few_nodes():
    # six boxes of 64^3, 128^3 and 192^3 (two each; neutrino masses 0 .. 0.6 eV):
    # one pm_batch per grid size, each pass one persistent kernel over its boxes
    boxes = synth.batched_boxes(6, n_hist=8, n_kbins=32)
    direct = batch.Batch(boxes, n_streams=1, autotune=False)
    direct.eager_step()
    direct.check()
    ref = _dv(direct)
    ref_bins = [it["pm"].bins() for it in direct.items]
    direct.close()
    # two sub-batches per grid size on their own streams: the same velocities
    b = batch.Batch(boxes, persistent=True, split=2)
    assert len(b.groups) == 6
    b.eager_step()
    b.check()
    for d0, d1 in zip(ref, _dv(b)):
        assert np.abs(d1 - d0).max() <= 1e-5 * np.abs(d0).max()
    b.close()
    b = batch.Batch(boxes, persistent=True, split=1)
    assert len(b.groups) == 3
    b.eager_step()
    b.check()
    got = _dv(b)
    for d0, d1, it, rb in zip(ref, got, b.items, ref_bins):
        scale = np.abs(d0).max()
        rms = np.sqrt(((d1 - d0) ** 2).mean()) / np.sqrt((d0 ** 2).mean())
        print(f"box N={it['w'].ngrid} M_nu={it['w'].m_nu_total}: max {np.abs(d1 - d0).max() / scale:.2e}, rms {rms:.2e}")
        assert np.abs(d1 - d0).max() <= 1e-5 * scale and rms <= 1e-6
        cnt, ks, ps = it["pm"].bins()
        assert np.array_equal(cnt, rb[0]) and np.allclose(ps, rb[2], rtol=1e-6, atol=0)
    # the captured step: a few launches per grid size, bit for bit the eager step
    per_step = b.launches_per_step()
    assert per_step <= 3 * 17
    b.reset_velocities()
    g = b.capture()
    assert g.nodes() <= per_step + 3 * 6 + 8
    b.reset_velocities()
    b.step()
    b.check()
    again = _dv(b)
    for d1, d2 in zip(got, again):
        assert np.array_equal(d1, d2)
    b.step()
    b.check()
    two = _dv(b)
    for d1, d2 in zip(got, two):
        assert np.allclose(d2, 2 * d1, rtol=1e-5, atol=1e-6 * np.abs(d1).max())
    b.close()
