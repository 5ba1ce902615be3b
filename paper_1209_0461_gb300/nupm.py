"""Thin ctypes binding of libnupm (include/nupm.h).

Argument marshalling only: every step of the kick runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (torch supplies device memory and the
stream); host tables are numpy arrays.  The binding raises if the library is
missing or a call fails; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnupm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "nupm.h")

PM_OK = 0
ERRORS = {-1: "PM_ERR_INVALID", -2: "PM_ERR_RANGE", -3: "PM_ERR_OVERFLOW", -4: "PM_ERR_CUDA",
          -5: "PM_ERR_ALLOC", -6: "PM_ERR_TIMEOUT", -7: "PM_ERR_ORDER", -8: "PM_ERR_UNSUPPORTED"}
PM_FP64, PM_FP32 = 0, 1
PM_I_FIT, PM_DECONV_CIC, PM_KEEP_DEPOSIT, PM_UNFUSED_DEPOSIT = 0x1, 0x2, 0x4, 0x8
PM_TMA_COLUMNS, PM_FUSED_GATHER, PM_SPECTRAL_GRADIENT, PM_RELATIVISTIC = 0x10, 0x20, 0x40, 0x80
PM_IC_MULTIPOLE = 0x100
FIELD_DEPOSIT, FIELD_DELTA_K, FIELD_ACC_X, FIELD_ACC_Y, FIELD_ACC_Z, FIELD_PHI = range(6)
MLP_FEATURES, MLP_WIDTH = 12, 128
STAGES = ["deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_fwd", "bins", "response", "green",
          "fft_z_inv", "fft_y_inv", "fft_x_inv", "interp", "drift"]


class PmParams(C.Structure):
    _fields_ = [("ngrid", C.c_int32), ("npart", C.c_int64), ("box", C.c_double),
                ("particle_mass", C.c_double), ("omega_cdm", C.c_double), ("omega_nu", C.c_double),
                ("h", C.c_double), ("m_nu_total_eV", C.c_double), ("n_species", C.c_int32),
                ("m_nu_eV", C.c_double * 3), ("a_init", C.c_double), ("n_kbins", C.c_int32),
                ("n_hist_max", C.c_int32), ("precision", C.c_int32), ("flags", C.c_uint32),
                ("iters", C.c_int32), ("quad_nodes", C.c_int32)]


class PMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libnupm.so (built in-tree by paper_1209_0461_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1209_0461_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, dp, i32, i64, d = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64, C.c_double
    sig = {
        "pm_default_params": (None, [C.POINTER(PmParams)]),
        "pm_init": (C.c_int, [C.POINTER(PmParams), dp, dp, vp, C.POINTER(vp)]),
        "pm_deposit": (C.c_int, [vp, vp]),
        "pm_nu_response": (C.c_int, [vp, d, dp, vp, i32, vp, vp, vp, vp]),
        "pm_nu_prepare": (C.c_int, [vp, d, dp, vp, i32]),
        "pm_kick": (C.c_int, [vp, vp, vp, d, d, vp]),
        "pm_check": (C.c_int, [vp]),
        "pm_free": (None, [vp]),
        "pm_last_error": (C.c_char_p, [vp]),
        "pm_kick_factor": (d, [vp, d, d]),
        "pm_drift_factor": (d, [vp, d, d]),
        "pm_hubble": (d, [C.POINTER(PmParams), d]),
        "pm_measure_fp64_fma": (C.c_int, [i32, dp, vp]),
        "pm_drift": (C.c_int, [vp, vp, vp, d]),
        "pm_history_set": (C.c_int, [vp, dp, vp, i32, vp]),
        "pm_history_get": (C.c_int, [vp, dp, vp, vp, C.POINTER(C.c_int32)]),
        "pm_step": (C.c_int, [vp, vp, vp, d, d, d, vp]),
        "pm_get_bins": (C.c_int, [vp, dp, dp, dp]),
        "pm_get_thresholds": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "pm_copy_field": (C.c_int, [vp, i32, vp]),
        "pm_device_bytes": (i64, [vp]),
        "pm_timing": (C.c_int, [vp, i32]),
        "pm_get_timing": (C.c_int, [vp, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "pm_bin_power_static": (C.c_int, [vp, i32, d, i32, i32, vp, vp, vp, vp]),
        "pm_mlp_create": (C.c_int, [i32, i32, vp, C.POINTER(vp)]),
        "pm_mlp_free": (None, [vp]),
        "pm_mlp_param_count": (i64, [vp]),
        "pm_mlp_set_params": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "pm_mlp_get_params": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "pm_mlp_set_norm": (C.c_int, [vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float]),
        "pm_mlp_forward": (C.c_int, [vp, vp, i64, vp]),
        "pm_mlp_grad": (C.c_int, [vp, vp, vp, i64, vp, vp]),
        "pm_mlp_train_step": (C.c_int, [vp, vp, vp, i64, C.c_float, vp]),
        "pm_response_features": (C.c_int, [vp, d, dp, vp, i32, vp]),
        "pm_nu_response_mlp": (C.c_int, [vp, vp, d, dp, vp, i32, vp, vp, vp]),
        "pm_set_power": (C.c_int, [vp, dp, dp, dp]),
        "pm_autotune": (C.c_int, [vp, vp, vp, d, dp, vp, i32, i32, C.POINTER(C.c_int32)]),
        "pm_set_tuning": (C.c_int, [vp, C.POINTER(C.c_int32)]),
        "pm_batch_create": (C.c_int, [C.POINTER(vp), i32, vp, C.POINTER(vp)]),
        "pm_batch_kick": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), dp, dp, C.POINTER(dp), C.POINTER(vp),
                                    C.POINTER(C.c_int32)]),
        "pm_batch_launches": (i64, [vp]),
        "pm_batch_last_error": (C.c_char_p, [vp]),
        "pm_batch_free": (None, [vp]),
        "pm_graph_begin": (C.c_int, [vp]),
        "pm_graph_end": (C.c_int, [vp, C.POINTER(vp)]),
        "pm_graph_launch": (C.c_int, [vp, vp]),
        "pm_graph_nodes": (i64, [vp]),
        "pm_graph_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_symbols():
    """Names of the functions include/nupm.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"NUPM_API\s+[\w\s\*]*?\b(pm_\w+)\s*\(", txt)))


def _dptr(arr):
    return arr.ctypes.data_as(C.POINTER(C.c_double)) if arr is not None else None


def _tptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def measure_fp64_fma(iters=256, stream=None):
    """pm_measure_fp64_fma: the device's FP64 FMA rate in TFLOP/s."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    rc = lib().pm_measure_fp64_fma(int(iters), C.byref(out), C.c_void_p(st.cuda_stream))
    if rc != PM_OK:
        raise PMError(rc, "pm_measure_fp64_fma failed")
    return out.value


def hubble(a, omega_cdm, omega_nu=-1.0, h=0.7, m_nu_total=0.0, n_species=3, m_nu=None, flags=0):
    """pm_hubble: H(a)/H0 of a problem statement's background, host only."""
    L = lib()
    p = PmParams()
    L.pm_default_params(C.byref(p))
    p.omega_cdm, p.omega_nu, p.h = float(omega_cdm), float(omega_nu), float(h)
    p.m_nu_total_eV, p.n_species = float(m_nu_total), int(n_species)
    for i, m in enumerate(m_nu or ()):
        p.m_nu_eV[i] = float(m)
    p.flags = int(flags)
    return float(L.pm_hubble(C.byref(p), float(a)))


def bin_power_static(spec, ngrid, box, n_kbins, count=None, ksum=None, psum=None, stream=None):
    """pm_bin_power_static: bins of a CUDA rfftn-layout spectrum (complex128 or
    complex64 [N, N, N/2+1]) into caller-given CUDA float64 [n_kbins] tensors,
    without any device allocation inside the library."""
    import torch
    if spec.dtype not in (torch.complex128, torch.complex64) or not spec.is_cuda or not spec.is_contiguous():
        raise ValueError("spec must be a contiguous CUDA complex tensor [N, N, N/2+1]")
    if tuple(spec.shape) != (ngrid, ngrid, ngrid // 2 + 1):
        raise ValueError("spec shape must be [N, N, N/2+1]")
    for t in (count, ksum, psum):
        if t is not None and (t.dtype != torch.float64 or not t.is_cuda or t.numel() < n_kbins):
            raise ValueError("outputs must be CUDA float64 [n_kbins]")
    for t in (count, ksum, psum):
        if t is not None and t.device != spec.device:
            raise ValueError("outputs must be on the spectrum's device")
    if stream is not None and stream.device != spec.device:
        raise ValueError("stream must be on the spectrum's device")
    prec = PM_FP64 if spec.dtype == torch.complex128 else PM_FP32
    with torch.cuda.device(spec.device):     # the library's scratch is the current device's
        st = stream if stream is not None else torch.cuda.current_stream(spec.device)
        rc = lib().pm_bin_power_static(_tptr(spec), int(ngrid), float(box), int(n_kbins), prec, _tptr(count),
                                       _tptr(ksum), _tptr(psum), C.c_void_p(st.cuda_stream))
    if rc != PM_OK:
        raise PMError(rc, "pm_bin_power_static failed")


class PM:
    """One PM context (pm_init .. pm_free) on the current CUDA device."""

    def __init__(self, ngrid, npart, box, omega_cdm, omega_nu=-1.0, h=0.7, m_nu_total=0.0,
                 n_species=3, m_nu=None, a_init=0.02, n_kbins=32, n_hist_max=128,
                 precision="fp64", flags=0, iters=1, quad_nodes=8, sqrtPnu_init=None,
                 theta_over_delta_init=None, stream=None, particle_mass=1.0):
        import torch
        L = lib()
        p = PmParams()
        L.pm_default_params(C.byref(p))
        p.ngrid, p.npart, p.box = int(ngrid), int(npart), float(box)
        p.particle_mass = float(particle_mass)
        p.omega_cdm, p.omega_nu, p.h = float(omega_cdm), float(omega_nu), float(h)
        p.m_nu_total_eV, p.n_species = float(m_nu_total), int(n_species)
        for i, m in enumerate(m_nu or ()):
            p.m_nu_eV[i] = float(m)
        p.a_init = float(a_init)
        p.n_kbins, p.n_hist_max = int(n_kbins), int(n_hist_max)
        p.precision = PM_FP64 if precision == "fp64" else PM_FP32
        p.flags, p.iters, p.quad_nodes = int(flags), int(iters), int(quad_nodes)
        self.params = p
        self.fp64 = p.precision == PM_FP64
        self.dtype = torch.float64 if self.fp64 else torch.float32
        self.nk = p.n_kbins
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        pi = None if sqrtPnu_init is None else np.ascontiguousarray(sqrtPnu_init, dtype=np.float64)
        ti = None if theta_over_delta_init is None else np.ascontiguousarray(
            theta_over_delta_init, dtype=np.float64)
        if m_nu_total <= 0 or n_species <= 0:
            pi = ti = None                     # no massive species: nothing to initialise
        for arr in (pi, ti):
            if arr is not None and arr.size < n_species * self.nk:
                raise ValueError("initial-condition arrays must hold n_species x n_kbins values")
        ctx = C.c_void_p()
        rc = L.pm_init(C.byref(p), _dptr(pi), _dptr(ti), C.c_void_p(self.stream.cuda_stream),
                       C.byref(ctx))
        if rc != PM_OK:
            raise PMError(rc, "pm_init failed (see stderr)")
        self.ctx = ctx

    # -- helpers
    def _ok(self, rc, what):
        if rc != PM_OK:
            raise PMError(rc, f"{what}: {lib().pm_last_error(self.ctx).decode()}")

    def _check_pos(self, pos):
        import torch
        n = self.params.npart
        if not pos.is_cuda or not pos.is_contiguous():
            raise ValueError("positions must be a contiguous CUDA tensor")
        if self.fp64:
            if pos.dtype != torch.float64 or tuple(pos.shape) != (3, n):
                raise ValueError("PM_FP64 positions: float64 tensor [3, npart]")
        elif pos.dtype != torch.int32 or tuple(pos.shape) != (6, n):
            raise ValueError("PM_FP32 positions: int32 tensor [6, npart] (cells, offset bits)")

    # -- the kick
    def deposit(self, pos):
        self._check_pos(pos)
        self._ok(lib().pm_deposit(self.ctx, _tptr(pos)), "pm_deposit")

    def nu_response(self, a, a_hist, sqrtPM_hist, sqrtPnu_prev=None, ratio=None, sqrtPnu=None,
                    sqrtPM=None):
        """a_hist: host array [n]; sqrtPM_hist: CUDA float64 [n, n_kbins] (or None for n = 0);
        outputs: optional CUDA float64 [n_kbins] tensors filled in place."""
        import torch
        ah = np.ascontiguousarray(a_hist if a_hist is not None else [], dtype=np.float64)
        n = int(ah.size)
        if n:
            if (sqrtPM_hist is None or sqrtPM_hist.dtype != torch.float64 or not sqrtPM_hist.is_cuda
                    or sqrtPM_hist.numel() < n * self.nk or not sqrtPM_hist.is_contiguous()):
                raise ValueError("sqrtPM_hist must be a contiguous CUDA float64 [n_hist, n_kbins]")
        for t in (sqrtPnu_prev, ratio, sqrtPnu, sqrtPM):
            if t is not None and (t.dtype != torch.float64 or not t.is_cuda or t.numel() < self.nk):
                raise ValueError("per-bin vectors must be CUDA float64 [n_kbins]")
        self._ok(lib().pm_nu_response(self.ctx, float(a), _dptr(ah) if n else None,
                                      _tptr(sqrtPM_hist) if n else None, n, _tptr(sqrtPnu_prev),
                                      _tptr(ratio), _tptr(sqrtPnu), _tptr(sqrtPM)), "pm_nu_response")

    def nu_prepare(self, a, a_hist, sqrtPM_hist):
        """pm_nu_prepare: launch the history panels of the next nu_response with
        the same arguments on the context's side stream (before deposit)."""
        ah, n = self._history(a_hist, sqrtPM_hist)
        self._ok(lib().pm_nu_prepare(self.ctx, float(a), _dptr(ah) if n else None,
                                     _tptr(sqrtPM_hist) if n else None, n), "pm_nu_prepare")

    def kick(self, pos, vel, a, kick_factor, acc_out=None):
        self._check_pos(pos)
        n = self.params.npart
        for t in (vel, acc_out):
            if t is not None and (t.dtype != self.dtype or tuple(t.shape) != (3, n) or not t.is_cuda
                                  or not t.is_contiguous()):
                raise ValueError(f"velocities / accelerations: contiguous CUDA {self.dtype} [3, npart]")
        self._ok(lib().pm_kick(self.ctx, _tptr(pos), _tptr(vel), float(a), float(kick_factor),
                               _tptr(acc_out)), "pm_kick")

    def check(self):
        self._ok(lib().pm_check(self.ctx), "pm_check")

    # -- the step loop (Sec. 4.3)
    def _check_vel(self, *ts):
        n = self.params.npart
        for t in ts:
            if t is not None and (t.dtype != self.dtype or tuple(t.shape) != (3, n) or not t.is_cuda
                                  or not t.is_contiguous()):
                raise ValueError(f"velocities / accelerations: contiguous CUDA {self.dtype} [3, npart]")

    def drift(self, pos, vel, drift_factor):
        """pm_drift: positions moved by vel * drift_factor, in place."""
        self._check_pos(pos)
        self._check_vel(vel)
        self._ok(lib().pm_drift(self.ctx, _tptr(pos), _tptr(vel), float(drift_factor)), "pm_drift")

    def history_set(self, a_hist, sqrtPM_hist, sqrtPnu_prev=None):
        """pm_history_set: the context's stored history (host a_hist [n], CUDA
        float64 [n, n_kbins]) and optional previous P_nu^{1/2} (CUDA [n_kbins])."""
        ah, n = self._history(a_hist, sqrtPM_hist)
        self._ok(lib().pm_history_set(self.ctx, _dptr(ah) if n else None, _tptr(sqrtPM_hist) if n else None, n,
                                      _tptr(sqrtPnu_prev)), "pm_history_set")

    def history_get(self):
        """(a_hist numpy [n], sqrtPM_hist CUDA float64 [n, n_kbins], sqrtPnu_prev CUDA [n_kbins] or None)."""
        import torch
        cnt = C.c_int32()
        self._ok(lib().pm_history_get(self.ctx, None, None, None, C.byref(cnt)), "pm_history_get")
        n = cnt.value
        ah = np.zeros(max(n, 1))
        rows = torch.zeros((max(n, 1), self.nk), dtype=torch.float64, device="cuda")
        prev = torch.full((self.nk,), float("nan"), dtype=torch.float64, device="cuda")
        self._ok(lib().pm_history_get(self.ctx, _dptr(ah), _tptr(rows), _tptr(prev), C.byref(cnt)), "pm_history_get")
        self.stream.synchronize()
        return ah[:n], rows[:n], (None if bool(torch.isnan(prev).all()) else prev)

    def step(self, pos, vel, a, kick_factor, drift_factor, acc_out=None):
        """pm_step: one Sec. 4.3 time step at a (deposit, response over the stored
        history, kick, store P_M, drift)."""
        self._check_pos(pos)
        self._check_vel(vel, acc_out)
        self._ok(lib().pm_step(self.ctx, _tptr(pos), _tptr(vel), float(a), float(kick_factor), float(drift_factor),
                               _tptr(acc_out)), "pm_step")

    def _history(self, a_hist, sqrtPM_hist):
        import torch
        ah = np.ascontiguousarray(a_hist if a_hist is not None else [], dtype=np.float64)
        n = int(ah.size)
        if n and (sqrtPM_hist is None or sqrtPM_hist.dtype != torch.float64 or not sqrtPM_hist.is_cuda
                  or sqrtPM_hist.numel() < n * self.nk or not sqrtPM_hist.is_contiguous()):
            raise ValueError("sqrtPM_hist must be a contiguous CUDA float64 [n_hist, n_kbins]")
        return ah, n

    # -- the learned response
    def response_features(self, a, a_hist, sqrtPM_hist, X=None):
        """pm_response_features -> CUDA float32 [n_kbins, 12]."""
        import torch
        ah, n = self._history(a_hist, sqrtPM_hist)
        if X is None:
            X = torch.empty((self.nk, MLP_FEATURES), dtype=torch.float32, device="cuda")
        elif X.dtype != torch.float32 or not X.is_cuda or X.numel() < self.nk * MLP_FEATURES:
            raise ValueError("X must be CUDA float32 [n_kbins, 12]")
        self._ok(lib().pm_response_features(self.ctx, float(a), _dptr(ah) if n else None,
                                            _tptr(sqrtPM_hist) if n else None, n, _tptr(X)),
                 "pm_response_features")
        return X

    def nu_response_mlp(self, mlp, a, a_hist, sqrtPM_hist, ratio=None, sqrtPnu=None, sqrtPM=None):
        """pm_nu_response_mlp: the surrogate in place of the response integral."""
        import torch
        ah, n = self._history(a_hist, sqrtPM_hist)
        for t in (ratio, sqrtPnu, sqrtPM):
            if t is not None and (t.dtype != torch.float64 or not t.is_cuda or t.numel() < self.nk):
                raise ValueError("per-bin vectors must be CUDA float64 [n_kbins]")
        self._ok(lib().pm_nu_response_mlp(self.ctx, mlp.handle, float(a), _dptr(ah) if n else None,
                                          _tptr(sqrtPM_hist) if n else None, n, _tptr(ratio), _tptr(sqrtPnu),
                                          _tptr(sqrtPM)), "pm_nu_response_mlp")

    def set_power(self, count, ksum, psum):
        """pm_set_power: host float64 [n_kbins] bins (units of bins())."""
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (count, ksum, psum)]
        if any(x.size != self.nk for x in arrs):
            raise ValueError("count, ksum, psum must hold n_kbins values")
        self._ok(lib().pm_set_power(self.ctx, *(_dptr(x) for x in arrs)), "pm_set_power")

    # -- tuning
    def autotune(self, pos, vel, a, a_hist, sqrtPM_hist, reps=2):
        """pm_autotune: returns (wide_y, wide_z, ctas_per_sm, gather_rows); wide_z = 2
        is the TMA-staged z pass, gather_rows = 1 the gather in the sort's row order,
        2 the same order with forces by sorted slot and the velocity update in
        particle order."""
        self._check_pos(pos)
        ah, n = self._history(a_hist, sqrtPM_hist)
        t = (C.c_int32 * 4)()
        self._ok(lib().pm_autotune(self.ctx, _tptr(pos), _tptr(vel), float(a), _dptr(ah) if n else None,
                                   _tptr(sqrtPM_hist) if n else None, n, int(reps), t), "pm_autotune")
        return tuple(int(x) for x in t)

    def set_tuning(self, wide_y=-1, wide_z=-1, ctas_per_sm=16, gather_rows=0):
        t = (C.c_int32 * 4)(int(wide_y), int(wide_z), int(ctas_per_sm), int(gather_rows))
        self._ok(lib().pm_set_tuning(self.ctx, t), "pm_set_tuning")

    # -- background
    def kick_factor(self, a0, a1):
        return lib().pm_kick_factor(self.ctx, float(a0), float(a1))

    def drift_factor(self, a0, a1):
        return lib().pm_drift_factor(self.ctx, float(a0), float(a1))

    # -- inspection
    def bins(self):
        cnt, ks, ps = (np.zeros(self.nk) for _ in range(3))
        self._ok(lib().pm_get_bins(self.ctx, _dptr(cnt), _dptr(ks), _dptr(ps)), "pm_get_bins")
        return cnt, ks, ps

    def thresholds(self):
        t = np.zeros(self.nk + 1, dtype=np.int64)
        self._ok(lib().pm_get_thresholds(self.ctx, t.ctypes.data_as(C.POINTER(C.c_int64))),
                 "pm_get_thresholds")
        return t

    def field(self, which):
        import torch
        n = self.params.ngrid
        if which == FIELD_DEPOSIT:
            out = torch.empty((n, n, n), dtype=torch.int64, device="cuda")
        elif which == FIELD_DELTA_K:
            out = torch.empty((n, n, n // 2 + 1), dtype=torch.complex128 if self.fp64 else torch.complex64,
                              device="cuda")
        else:
            out = torch.empty((n, n, n), dtype=self.dtype, device="cuda")
        self._ok(lib().pm_copy_field(self.ctx, int(which), _tptr(out)), "pm_copy_field")
        return out

    def timing(self, enable=True):
        """Start (clear) or stop per-stage CUDA-event timing."""
        self._ok(lib().pm_timing(self.ctx, 1 if enable else 0), "pm_timing")

    def get_timing(self):
        """{stage: (total ms, kernel launches, calls)} since timing(True)."""
        ms = np.zeros(len(STAGES))
        ln = np.zeros(len(STAGES), dtype=np.int64)
        ca = np.zeros(len(STAGES), dtype=np.int64)
        self._ok(lib().pm_get_timing(self.ctx, _dptr(ms), ln.ctypes.data_as(C.POINTER(C.c_int64)),
                                     ca.ctypes.data_as(C.POINTER(C.c_int64))), "pm_get_timing")
        return {name: (float(ms[i]), int(ln[i]), int(ca[i])) for i, name in enumerate(STAGES)}

    def device_bytes(self):
        return int(lib().pm_device_bytes(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            lib().pm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The surrogate network (pm_mlp_*): 12 -> 128 -> 128 -> 1, tanh, BF16 weights."""

    def __init__(self, n_in=MLP_FEATURES, width=MLP_WIDTH, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = lib().pm_mlp_create(int(n_in), int(width), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != PM_OK:
            raise PMError(rc, "pm_mlp_create failed")
        self.handle = h
        self.n_in = int(n_in)
        self.P = int(lib().pm_mlp_param_count(h))

    def _ok(self, rc, what):
        if rc != PM_OK:
            raise PMError(rc, what)

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != self.P:
            raise ValueError(f"expected {self.P} parameters")
        self._ok(lib().pm_mlp_set_params(self.handle, th.ctypes.data_as(C.POINTER(C.c_float))), "pm_mlp_set_params")

    def get_params(self):
        th = np.zeros(self.P, dtype=np.float32)
        self._ok(lib().pm_mlp_get_params(self.handle, th.ctypes.data_as(C.POINTER(C.c_float))), "pm_mlp_get_params")
        return th

    def set_norm(self, mu, sigma, y_mu, y_sigma):
        m = np.ascontiguousarray(mu, dtype=np.float32)
        s = np.ascontiguousarray(sigma, dtype=np.float32)
        if m.size != self.n_in or s.size != self.n_in:
            raise ValueError("mu and sigma need n_in values")
        self._ok(lib().pm_mlp_set_norm(self.handle, m.ctypes.data_as(C.POINTER(C.c_float)),
                                       s.ctypes.data_as(C.POINTER(C.c_float)), float(y_mu), float(y_sigma)),
                 "pm_mlp_set_norm")
        self.norm = (m.astype(np.float64), s.astype(np.float64), float(np.float32(y_mu)), float(np.float32(y_sigma)))

    def _xy(self, X, y=None):
        import torch
        if X.dtype != torch.float32 or not X.is_cuda or not X.is_contiguous() or X.dim() != 2 or X.shape[1] != self.n_in:
            raise ValueError("X must be a contiguous CUDA float32 [n, n_in]")
        if y is not None and (y.dtype != torch.float32 or not y.is_cuda or y.numel() != X.shape[0]):
            raise ValueError("y must be CUDA float32 [n]")
        return int(X.shape[0])

    def forward(self, X, out=None):
        import torch
        n = self._xy(X)
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device="cuda")
        self._ok(lib().pm_mlp_forward(self.handle, _tptr(X), n, _tptr(out)), "pm_mlp_forward")
        return out

    def grad(self, X, y):
        """(grad CUDA float32 [P], loss CUDA float32 [1])."""
        import torch
        n = self._xy(X, y)
        g = torch.empty(self.P, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._ok(lib().pm_mlp_grad(self.handle, _tptr(X), _tptr(y), n, _tptr(g), _tptr(loss)), "pm_mlp_grad")
        return g, loss

    def train_step(self, X, y, lr, loss=None):
        n = self._xy(X, y)
        self._ok(lib().pm_mlp_train_step(self.handle, _tptr(X), _tptr(y), n, float(lr), _tptr(loss)),
                 "pm_mlp_train_step")

    def close(self):
        if getattr(self, "handle", None):
            lib().pm_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured CUDA graph of pm_* calls (pm_graph_begin .. pm_graph_end)."""

    def __init__(self, handle):
        self.handle = handle

    @staticmethod
    def capture(stream, fn):
        """Capture everything fn() issues on `stream` (and streams joined to it)."""
        L = lib()
        rc = L.pm_graph_begin(C.c_void_p(stream.cuda_stream))
        if rc != PM_OK:
            raise PMError(rc, "pm_graph_begin")
        try:
            fn()
        finally:
            h = C.c_void_p()
            rc = L.pm_graph_end(C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != PM_OK:
            raise PMError(rc, "pm_graph_end")
        return Graph(h)

    def launch(self, stream):
        rc = lib().pm_graph_launch(self.handle, C.c_void_p(stream.cuda_stream))
        if rc != PM_OK:
            raise PMError(rc, "pm_graph_launch")

    def nodes(self):
        return int(lib().pm_graph_nodes(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().pm_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPM:
    """pm_batch: contexts of one grid size kicked together, one persistent
    kernel per pass over all boxes (work taken from an atomic counter)."""

    def __init__(self, contexts, stream=None):
        import torch
        self.contexts = list(contexts)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (C.c_void_p * len(self.contexts))(*[pm.ctx.value for pm in self.contexts])
        out = C.c_void_p()
        rc = lib().pm_batch_create(arr, len(self.contexts), C.c_void_p(self.stream.cuda_stream), C.byref(out))
        if rc != PM_OK:
            raise PMError(rc, "pm_batch_create failed (see stderr)")
        self.b = out

    def launches(self):
        return int(lib().pm_batch_launches(self.b))

    def kick(self, pos, vel, a, kick_factor, a_hist=None, sqrtPM_hist=None):
        """pos, vel: lists of CUDA tensors (one per box); a, kick_factor: per box;
        a_hist: list of host arrays (or None); sqrtPM_hist: list of CUDA float64
        [n, n_kbins] tensors (or None)."""
        nb = len(self.contexts)
        vp = C.c_void_p
        P = (vp * nb)(*[C.c_void_p(t.data_ptr()) for t in pos])
        V = (vp * nb)(*[C.c_void_p(t.data_ptr()) for t in vel])
        A = np.ascontiguousarray(a, dtype=np.float64)
        K = np.ascontiguousarray(kick_factor, dtype=np.float64)
        keep = []
        ah_p = (C.POINTER(C.c_double) * nb)()
        h_p = (vp * nb)()
        nh = (C.c_int32 * nb)()
        for i in range(nb):
            ah = None if a_hist is None else a_hist[i]
            if ah is not None and len(ah):
                arr = np.ascontiguousarray(ah, dtype=np.float64)
                keep.append(arr)
                ah_p[i] = arr.ctypes.data_as(C.POINTER(C.c_double))
                h_p[i] = C.c_void_p(sqrtPM_hist[i].data_ptr())
                nh[i] = len(arr)
        self._keep = keep          # host arrays stay alive (and unchanged) for a captured graph
        rc = lib().pm_batch_kick(self.b, P, V, _dptr(A), _dptr(K), ah_p, h_p, nh)
        if rc != PM_OK:
            raise PMError(rc, lib().pm_batch_last_error(self.b).decode())

    def close(self):
        if self.b:
            lib().pm_batch_free(self.b)
            self.b = None
