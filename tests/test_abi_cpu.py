"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every function include/nupm.h declares, and rejects bad arguments
before touching the device."""
import ctypes as C

import pytest

from paper_1209_0461_gb300 import nupm


@pytest.fixture(scope="module")
def L():
    from paper_1209_0461_gb300 import build as b
    b.build()
    return nupm.lib()


def test_exports_every_declared_symbol(L):
    names = nupm.declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n


def test_params_struct_layout(L):
    p = nupm.PmParams()
    L.pm_default_params(C.byref(p))
    assert C.sizeof(p) == 128
    assert (p.ngrid, p.iters, p.quad_nodes, p.precision) == (32, 1, 8, nupm.PM_FP64)


@pytest.mark.parametrize("field,value,code", [
    ("ngrid", 17, -8), ("ngrid", 2048, -8), ("npart", 0, -1), ("box", -1.0, -1),
    ("omega_cdm", 0.0, -1), ("a_init", 0.0, -2), ("n_kbins", 0, -1), ("iters", 0, -1),
    ("quad_nodes", 1, -1), ("precision", 7, -1), ("m_nu_total_eV", -0.1, -2), ("flags", 0x200, -1),
])
def test_host_validation_without_gpu(L, field, value, code):
    p = nupm.PmParams()
    L.pm_default_params(C.byref(p))
    setattr(p, field, value)
    ctx = C.c_void_p(123)
    assert L.pm_init(C.byref(p), None, None, None, C.byref(ctx)) == code
    assert ctx.value is None


def test_null_arguments(L):
    assert L.pm_init(None, None, None, None, None) == -1
    assert L.pm_deposit(None, None) == -1
    assert L.pm_check(None) == -1
    assert L.pm_get_timing(None, None, None, None) == -1
    L.pm_free(None)
    assert L.pm_last_error(None) == b"null context"


def test_surrogate_entry_points_validate_without_gpu(L):
    h = C.c_void_p()
    assert L.pm_mlp_create(0, 128, None, C.byref(h)) == -1
    assert L.pm_mlp_create(12, 64, None, C.byref(h)) == -1
    assert L.pm_mlp_create(17, 128, None, C.byref(h)) == -1
    assert not h.value
    assert L.pm_mlp_param_count(None) == 0
    assert L.pm_mlp_forward(None, None, 4, None) == -1
    assert L.pm_mlp_train_step(None, None, None, 4, 0.1, None) == -1
    assert L.pm_set_power(None, None, None, None) == -1
    assert L.pm_response_features(None, 0.1, None, None, 0, None) == -1
    assert L.pm_nu_response_mlp(None, None, 0.1, None, None, 0, None, None, None) == -1


@pytest.mark.parametrize("masses", [(0.1, 0.1, 0.1), (0.022, 0.024, 0.054), (0.06,), ()])
def test_host_background_against_the_oracle(L, masses):
    # pm_hubble (host only, no GPU): matter + Lambda, and the Sec. 4.4
    # background of Eq. relativistic with radiation, against the oracle's
    # H(a) (its own quadrature of the Fermi-Dirac energy density)
    from oracle import pm_oracle as O
    from paper_1209_0461_gb300 import nupm
    h, om = 0.7, 0.3
    tot = sum(masses)
    onu = tot / (93.14 * h * h)
    for rel in (False, True):
        cos = O.Cosmo(om - onu, onu, h, tuple(masses), 0.02, relativistic=rel)
        for a in (1e-6, 1e-3, 0.02, 0.1, 0.5, 1.0, 2.0):
            got = nupm.hubble(a, om - onu, -1.0, h, tot, len(masses), list(masses),
                              flags=nupm.PM_RELATIVISTIC if rel else 0)
            want = float(O.hubble(a, cos))
            assert abs(got / want - 1) < (1e-15 if not rel else 2e-12), (rel, a, got, want)


def test_step_batch_and_peak_entry_points_validate_without_gpu(L):
    # the step loop, the persistent batch and the FP64 peak reject missing
    # arguments on the host, before any device work
    assert L.pm_drift(None, None, None, 0.1) == -1
    assert L.pm_history_set(None, None, None, 0, None) == -1
    assert L.pm_history_get(None, None, None, None, None) == -1
    assert L.pm_step(None, None, None, 0.1, 0.01, 0.01, None) == -1
    out = C.c_void_p(123)
    assert L.pm_batch_create(None, 0, None, C.byref(out)) == -1
    assert out.value is None
    assert L.pm_batch_create(None, 1, None, None) == -1
    assert L.pm_batch_kick(None, None, None, None, None, None, None, None) == -1
    assert L.pm_batch_launches(None) == 0
    assert L.pm_batch_last_error(None) == b"null batch"
    L.pm_batch_free(None)
    t = C.c_double(-1.0)
    assert L.pm_measure_fp64_fma(0, C.byref(t), None) == -1
    assert L.pm_measure_fp64_fma(8, None, None) == -1
