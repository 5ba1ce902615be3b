"""Failure paths of the C ABI on a GPU, injected on the host (no device fault).

NUPM_FAIL_ALLOC_AT=k makes the k-th device allocation of pm_init report
failure: for every k up to the last allocation pm_init must return
PM_ERR_ALLOC, hand back no context, and free everything it had allocated (the
device's free memory returns to where it was), and the next pm_init must
work."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_common import build_lib  # noqa: E402
from paper_1209_0461_gb300 import nupm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build_lib()


def _init(L, p):
    ctx = C.c_void_p()
    rc = L.pm_init(C.byref(p), None, None, None, C.byref(ctx))
    return rc, ctx


@pytest.mark.parametrize("prec", [nupm.PM_FP64, nupm.PM_FP32])
def test_every_failed_allocation_of_pm_init_is_cleaned_up(prec, monkeypatch):
    L = nupm.lib()
    p = nupm.PmParams()
    L.pm_default_params(C.byref(p))
    p.ngrid, p.npart, p.box = 256, 64 ** 3, 512.0
    p.omega_cdm, p.omega_nu, p.h = 0.29, -1.0, 0.7
    p.m_nu_total_eV, p.n_species = 0.3, 3
    p.precision = prec
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(1, 200):
        monkeypatch.setenv("NUPM_FAIL_ALLOC_AT", str(k))
        rc, ctx = _init(L, p)
        if rc == nupm.PM_OK:                # k is past the last allocation
            L.pm_free(ctx)
            break
        assert rc == -5, (k, rc)            # PM_ERR_ALLOC
        assert not ctx.value
        failed += 1
    else:
        pytest.fail("pm_init never succeeded")
    assert failed >= 20                     # every grid, table and buffer was a failure point
    monkeypatch.delenv("NUPM_FAIL_ALLOC_AT")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # one leaked spectrum alone would be 134 MB (FP64) / 67 MB (FP32)
    assert free0 - free1 < 8 << 20, (free0, free1)
    rc, ctx = _init(L, p)
    assert rc == nupm.PM_OK
    assert L.pm_device_bytes(ctx) > 4 * 256 ** 2 * 128 * (8 if prec == nupm.PM_FP32 else 16)
    L.pm_free(ctx)
