"""Thin ctypes binding of libtc (include/tc.h), argument marshalling only.

Every computation runs in libtc's CUDA kernels.  The functions below keep the
C names; ``Run`` wraps one context.  Spectral states are complex128 arrays of
shape (nfields, Nr, M+1, 2K+1): NumPy arrays are passed as host pointers,
CUDA torch tensors as device pointers.  There is no CPU fallback: importing
this module without a built ``libtc.so`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TC_LIB=debug loads the debug build (index checks, tc_debug_flags)
LIB_PATH = os.path.join(_HERE, "libtc_debug.so" if os.environ.get("TC_LIB") == "debug"
                        else "libtc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtc.so is not built ({LIB_PATH}); run __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "TC_OK", 1: "TC_ERR_ARG", 2: "TC_ERR_CUDA", 3: "TC_ERR_OOM",
          4: "TC_ERR_NONFINITE", 5: "TC_ERR_CFL", 6: "TC_ERR_STATE",
          7: "TC_ERR_TIMEOUT", 8: "TC_ERR_UNSUPPORTED"}


class TCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        msg = _lib.tc_status_string(status).decode()
        super().__init__(f"{where}: {self.name} ({msg})")


class tc_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("t", "dt", "E", "E_pert", "torque_i", "torque_o", "P_wall", "eps",
                 "buoy_work", "Nu_i", "Nu_o", "div_max", "div_rms", "cfl", "corr_diff")]


class tc_info(ctypes.Structure):
    _fields_ = [("Nr", ctypes.c_int), ("Ntheta", ctypes.c_int), ("Nz", ctypes.c_int),
                ("M", ctypes.c_int), ("K", ctypes.c_int), ("nfields", ctypes.c_int),
                ("coeffs_per_field", ctypes.c_longlong), ("state_bytes", ctypes.c_longlong),
                ("device_bytes", ctypes.c_size_t), ("launches", ctypes.c_longlong),
                ("tile_mb", ctypes.c_int), ("tile_lb", ctypes.c_int),
                ("tile_mbf", ctypes.c_int), ("tensor_theta", ctypes.c_int),
                ("tensor_z", ctypes.c_int)]


class tc_params(ctypes.Structure):
    _fields_ = [("Nr", ctypes.c_int), ("Ntheta", ctypes.c_int), ("Nz", ctypes.c_int),
                ("eta", ctypes.c_double), ("Lz", ctypes.c_double), ("Re_i", ctypes.c_double),
                ("Re_o", ctypes.c_double), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
                ("precision", ctypes.c_int)]


class tc_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "tc_create": [_I, _I, _I, _D, _D, _D, _D, _D, _D, ctypes.POINTER(_P)],
    "tc_destroy": [_P],
    "tc_set_option": [_P, ctypes.c_char_p, _D],
    "tc_set_stream": [_P, _P],
    "tc_get_info": [_P, ctypes.POINTER(tc_info)],
    "tc_set_state": [_P, _P, _I],
    "tc_set_state_regrid": [_P, _P, _I, _I, _I, _I, _D, _D, _I],
    "tc_get_state": [_P, _P, _I],
    "tc_get_pressure": [_P, _P, _I],
    "tc_init_perturbation": [_P, _P, _I, _I, _D, _P, _D],
    "tc_step": [_P, _I, _D, _P],
    "tc_get_clock": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "tc_set_clock": [_P, _D, _D],
    "tc_diagnostics": [_P, ctypes.POINTER(tc_diag)],
    "tc_nonlinear": [_P, _P, _P, _P],
    "tc_stage_solve": [_P, _P, _D, _P, _P],
    "tc_get_timing": [_P, _P, _I, ctypes.POINTER(_I)],
    "tc_reset_timing": [_P],
    "tc_nonlinear_noalloc": [_I, _I, _I, _D, _D, _D, _D, _P, _P, _P, _P],
    "tc_measure_fp64_rate": [_D, _P, ctypes.POINTER(_D)],
    "tc_adjoint_step": [_P, _P, _D, _P],
    "tc_record_bytes_per_step": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "tc_step_record": [_P, _I, _D, _P, ctypes.c_longlong],
    "tc_adjoint_steps": [_P, _I, _P, _D, _P],
    "tc_nonlinear_adjoint": [_P, _P, _P, _P],
    "tc_stage_solve_adjoint": [_P, _P, _D, _P],
    "tc_objective": [_P, ctypes.POINTER(_D), _P],
    "tc_init_perturbation_adjoint": [_P, _P, _I, _I, _P, _P],
    "tc_get_ic_scales": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "tc_ensemble_create": [_I, _P, _I, ctypes.POINTER(_P)],
    "tc_ensemble_member": [_P, _I, ctypes.POINTER(_P)],
    "tc_ensemble_step": [_P, _I, _P],
    "tc_ensemble_kernels_per_step": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "tc_ensemble_set_mode": [_P, _I],
    "tc_ensemble_get_mode": [_P, ctypes.POINTER(_I)],
    "tc_ensemble_destroy": [_P],
    "tc_autotune": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "tc_debug_flags": [ctypes.POINTER(ctypes.c_uint), _I],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.tc_status_string.argtypes = [ctypes.c_int]
_lib.tc_status_string.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["tc_status_string"])


def _check(st: int, where: str):
    if st != 0:
        raise TCError(st, where)


def _ptr(a):
    """(pointer, where) of a NumPy array (host, 0) or CUDA tensor (device, 1)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1
    raise TypeError("expected a NumPy array or a CUDA tensor")


def _sized(a, n: int, what: str, device_only: bool = False):
    """(pointer, where) of a complex128 array or tensor holding at least n
    entries; raises ValueError before any call when it does not, so a short
    or mistyped buffer never reaches a kernel or a host copy."""
    p, where = _ptr(a)
    if device_only and where != 1:
        raise ValueError(f"{what}: expected a CUDA tensor (device pointer)")
    dt = a.dtype
    ok = (dt == np.complex128) if isinstance(a, np.ndarray) else (str(dt) == "torch.complex128")
    if not ok:
        raise ValueError(f"{what}: expected complex128, got {dt}")
    numel = a.size if isinstance(a, np.ndarray) else a.numel()
    if numel < n:
        raise ValueError(f"{what}: {numel} entries, {n} needed")
    return p, where


def _state_len(ctx) -> int:
    i = tc_info()
    _check(_lib.tc_get_info(ctx, ctypes.byref(i)), "tc_get_info")
    return int(i.nfields) * int(i.coeffs_per_field)


def _plane_len(ctx) -> int:
    i = tc_info()
    _check(_lib.tc_get_info(ctx, ctypes.byref(i)), "tc_get_info")
    return int(i.coeffs_per_field)


# -- C names ------------------------------------------------------------------
def tc_create(Nr, Ntheta, Nz, eta, Lz, Re_i, Re_o=0.0, Ra=0.0, Pr=1.0):
    h = _P()
    _check(_lib.tc_create(Nr, Ntheta, Nz, eta, Lz, Re_i, Re_o, Ra, Pr, ctypes.byref(h)),
           "tc_create")
    return h


def tc_destroy(ctx):
    _check(_lib.tc_destroy(ctx), "tc_destroy")


def tc_set_option(ctx, key: str, value: float):
    _check(_lib.tc_set_option(ctx, key.encode(), float(value)), f"tc_set_option({key})")


def tc_set_stream(ctx, stream_ptr: int):
    _check(_lib.tc_set_stream(ctx, stream_ptr), "tc_set_stream")


def tc_get_info(ctx) -> tc_info:
    i = tc_info()
    _check(_lib.tc_get_info(ctx, ctypes.byref(i)), "tc_get_info")
    return i


def tc_set_state(ctx, spec):
    p, where = _sized(spec, _state_len(ctx), "tc_set_state")
    _check(_lib.tc_set_state(ctx, p, where), "tc_set_state")


def tc_set_state_regrid(ctx, spec, eta_src, Lz_src):
    """spec: state of another resolution, (nfields, Nr, M+1, 2K+1) complex128
    (numpy array or CUDA tensor); the sizes are read from its shape."""
    nf, Nr, M1, NK = spec.shape
    p, where = _sized(spec, nf * Nr * M1 * NK, "tc_set_state_regrid")
    _check(_lib.tc_set_state_regrid(ctx, p, int(Nr), int(M1 - 1), int((NK - 1) // 2), int(nf),
                                    float(eta_src), float(Lz_src), where),
           "tc_set_state_regrid")


def tc_get_state(ctx, out):
    p, where = _sized(out, _state_len(ctx), "tc_get_state")
    _check(_lib.tc_get_state(ctx, p, where), "tc_get_state")
    return out


def tc_get_pressure(ctx, out):
    p, where = _sized(out, _plane_len(ctx), "tc_get_pressure")
    _check(_lib.tc_get_pressure(ctx, p, where), "tc_get_pressure")
    return out


def tc_init_perturbation(ctx, psi, amp, tcoef=None, amp_T=0.0):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    mp, kp = psi.shape[1] - 1, (psi.shape[2] - 1) // 2
    tptr = None
    if tcoef is not None:
        tcoef = np.ascontiguousarray(tcoef, dtype=np.complex128)
        tptr = tcoef.ctypes.data
    _check(_lib.tc_init_perturbation(ctx, psi.ctypes.data, mp, kp, float(amp), tptr,
                                     float(amp_T)), "tc_init_perturbation")


def tc_step(ctx, nsteps: int, dt: float):
    used = np.zeros(max(nsteps, 1), dtype=np.float64)
    _check(_lib.tc_step(ctx, int(nsteps), float(dt), used.ctypes.data), "tc_step")
    return used[:nsteps]


def tc_get_clock(ctx):
    """(t, dt_prev): simulated time and the step the next dynamic step is
    compared with."""
    t, dtp = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.tc_get_clock(ctx, ctypes.byref(t), ctypes.byref(dtp)), "tc_get_clock")
    return t.value, dtp.value


def tc_set_clock(ctx, t: float, dt_prev: float):
    _check(_lib.tc_set_clock(ctx, float(t), float(dt_prev)), "tc_set_clock")


def tc_diagnostics(ctx) -> dict:
    d = tc_diag()
    _check(_lib.tc_diagnostics(ctx, ctypes.byref(d)), "tc_diagnostics")
    return {n: getattr(d, n) for n, _ in tc_diag._fields_}


def tc_nonlinear(ctx, state_dev, n_dev) -> float:
    rate = ctypes.c_double(0.0)
    n = _state_len(ctx)
    _check(_lib.tc_nonlinear(ctx, _sized(state_dev, n, "tc_nonlinear state", True)[0],
                             _sized(n_dev, n, "tc_nonlinear out", True)[0], ctypes.byref(rate)),
           "tc_nonlinear")
    return rate.value


def tc_stage_solve(ctx, rhs_dev, dt, x_out_dev, p_out_dev=None):
    n = _state_len(ctx)
    pp = (_sized(p_out_dev, _plane_len(ctx), "tc_stage_solve p_out", True)[0]
          if p_out_dev is not None else None)
    _check(_lib.tc_stage_solve(ctx, _sized(rhs_dev, n, "tc_stage_solve rhs", True)[0],
                               float(dt), _sized(x_out_dev, n, "tc_stage_solve x_out", True)[0],
                               pp), "tc_stage_solve")


def tc_get_timing(ctx) -> dict:
    """{kernel name: (launches, total ms)} recorded while option "timing" is 1."""
    n = _I(0)
    _check(_lib.tc_get_timing(ctx, None, 0, ctypes.byref(n)), "tc_get_timing")
    arr = (tc_kernel_time * max(n.value, 1))()
    _check(_lib.tc_get_timing(ctx, arr, n.value, ctypes.byref(n)), "tc_get_timing")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(n.value)}


def tc_reset_timing(ctx):
    _check(_lib.tc_reset_timing(ctx), "tc_reset_timing")


def tc_nonlinear_noalloc(Nr, Ntheta, Nz, eta, Lz, Ra, Pr, state_dev, n_dev, stream_ptr=None):
    """Nonlinear terms with no device allocation (fixed 32 MiB static scratch).

    For callers that cannot call cudaMalloc; see include/tc.h for the limits
    and for why overlapping calls must be serialised.  Returns the CFL rate.
    """
    rate = ctypes.c_double(0.0)
    nf = 4 if Ra != 0.0 else 3
    n = nf * int(Nr) * ((int(Ntheta) - 1) // 3 + 1) * (2 * ((int(Nz) - 1) // 3) + 1)
    _check(_lib.tc_nonlinear_noalloc(int(Nr), int(Ntheta), int(Nz), float(eta), float(Lz),
                                     float(Ra), float(Pr),
                                     _sized(state_dev, n, "tc_nonlinear_noalloc state", True)[0],
                                     _sized(n_dev, n, "tc_nonlinear_noalloc out", True)[0],
                                     stream_ptr, ctypes.byref(rate)), "tc_nonlinear_noalloc")
    return rate.value


def tc_measure_fp64_rate(target_ms=250.0, stream_ptr=None):
    """Sustained FP64 FMA rate of the current device in TFLOP/s (a measurement
    aid for the ALU roofline; see include/tc.h)."""
    out = ctypes.c_double(0.0)
    _check(_lib.tc_measure_fp64_rate(float(target_ms), stream_ptr, ctypes.byref(out)),
           "tc_measure_fp64_rate")
    return out.value


def tc_adjoint_step(ctx, state_n_dev, dt, adj_dev):
    """adj <- P_H J(state_n)^T adj for one step at fixed dt (in place)."""
    n = _state_len(ctx)
    _check(_lib.tc_adjoint_step(ctx, _sized(state_n_dev, n, "tc_adjoint_step state", True)[0],
                                float(dt), _sized(adj_dev, n, "tc_adjoint_step adj", True)[0]),
           "tc_adjoint_step")


def tc_record_bytes_per_step(ctx) -> int:
    b = ctypes.c_longlong(0)
    _check(_lib.tc_record_bytes_per_step(ctx, ctypes.byref(b)), "tc_record_bytes_per_step")
    return b.value


def tc_step_record(ctx, nsteps, dt, record_dev):
    """record_dev: CUDA tensor of at least nsteps * tc_record_bytes_per_step bytes."""
    if not getattr(record_dev, "is_cuda", False):
        raise ValueError("tc_step_record: record_dev must be a CUDA tensor")
    nbytes = record_dev.numel() * record_dev.element_size()
    _check(_lib.tc_step_record(ctx, int(nsteps), float(dt), _ptr(record_dev)[0], int(nbytes)),
           "tc_step_record")


def tc_adjoint_steps(ctx, nsteps, record_dev, dt, adj_dev):
    need = int(nsteps) * tc_record_bytes_per_step(ctx)
    if not getattr(record_dev, "is_cuda", False) or \
            record_dev.numel() * record_dev.element_size() < need:
        raise ValueError(f"tc_adjoint_steps: a CUDA tensor of at least {need} bytes needed")
    _check(_lib.tc_adjoint_steps(ctx, int(nsteps), _ptr(record_dev)[0], float(dt),
                                 _sized(adj_dev, _state_len(ctx), "tc_adjoint_steps adj",
                                        True)[0]), "tc_adjoint_steps")


def tc_nonlinear_adjoint(ctx, state_dev, nbar_dev, xbar_dev):
    n = _state_len(ctx)
    _check(_lib.tc_nonlinear_adjoint(ctx, _sized(state_dev, n, "state", True)[0],
                                     _sized(nbar_dev, n, "nbar", True)[0],
                                     _sized(xbar_dev, n, "xbar", True)[0]),
           "tc_nonlinear_adjoint")


def tc_stage_solve_adjoint(ctx, xbar_dev, dt, rbar_dev):
    n = _state_len(ctx)
    _check(_lib.tc_stage_solve_adjoint(ctx, _sized(xbar_dev, n, "xbar", True)[0], float(dt),
                                       _sized(rbar_dev, n, "rbar", True)[0]),
           "tc_stage_solve_adjoint")


def tc_objective(ctx, grad_dev=None) -> float:
    J = ctypes.c_double(0.0)
    gp = (_sized(grad_dev, _state_len(ctx), "tc_objective grad", True)[0]
          if grad_dev is not None else None)
    _check(_lib.tc_objective(ctx, ctypes.byref(J), gp), "tc_objective")
    return J.value


def tc_init_perturbation_adjoint(ctx, lam_dev, mp, kp, with_T=False):
    pb = np.zeros((3, mp + 1, 2 * kp + 1), dtype=np.complex128)
    tb = np.zeros((mp + 1, 2 * kp + 1), dtype=np.complex128) if with_T else None
    lp = _sized(lam_dev, _state_len(ctx), "tc_init_perturbation_adjoint lam", True)[0]
    _check(_lib.tc_init_perturbation_adjoint(ctx, lp, int(mp), int(kp),
                                             pb.ctypes.data,
                                             tb.ctypes.data if tb is not None else None),
           "tc_init_perturbation_adjoint")
    return pb, tb


def tc_get_ic_scales(ctx):
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.tc_get_ic_scales(ctx, ctypes.byref(a), ctypes.byref(b)), "tc_get_ic_scales")
    return a.value, b.value


def tc_ensemble_create(workloads, autotune_tiles=True):
    n = len(workloads)
    arr = (tc_params * n)()
    for i, w in enumerate(workloads):
        arr[i] = tc_params(w.Nr, w.Ntheta, w.Nz, w.eta, w.Lz, w.Re_i, w.Re_o, w.Ra, w.Pr,
                           int(getattr(w, "precision", 0)))
    h = _P()
    _check(_lib.tc_ensemble_create(n, ctypes.cast(arr, _P), int(bool(autotune_tiles)),
                                   ctypes.byref(h)), "tc_ensemble_create")
    return h


def tc_ensemble_member(ens, i):
    h = _P()
    _check(_lib.tc_ensemble_member(ens, int(i), ctypes.byref(h)), "tc_ensemble_member")
    return h


def tc_ensemble_step(ens, nsteps, dts):
    d = np.ascontiguousarray(dts, dtype=np.float64)
    _check(_lib.tc_ensemble_step(ens, int(nsteps), d.ctypes.data), "tc_ensemble_step")


def tc_ensemble_set_mode(ens, mode: int):
    """0 graph of per-member kernels (default), 1 persistent kernel, 2 the
    persistent kernel's timeout test hook (see include/tc.h)."""
    _check(_lib.tc_ensemble_set_mode(ens, int(mode)), "tc_ensemble_set_mode")


def tc_ensemble_get_mode(ens) -> int:
    m = _I(0)
    _check(_lib.tc_ensemble_get_mode(ens, ctypes.byref(m)), "tc_ensemble_get_mode")
    return m.value


def tc_ensemble_kernels_per_step(ens):
    n = ctypes.c_longlong(0)
    _check(_lib.tc_ensemble_kernels_per_step(ens, ctypes.byref(n)), "tc_ensemble_kernels_per_step")
    return n.value


def tc_autotune(ctx):
    a, b = _I(0), _I(0)
    _check(_lib.tc_autotune(ctx, ctypes.byref(a), ctypes.byref(b)), "tc_autotune")
    return a.value, b.value


def tc_ensemble_destroy(ens):
    _check(_lib.tc_ensemble_destroy(ens), "tc_ensemble_destroy")


def tc_debug_flags(clear=False) -> int:
    """Check-site bits of the debug build's index checks (see include/tc.h);
    raises TCError (TC_ERR_UNSUPPORTED) in the normal build."""
    f = ctypes.c_uint(0)
    _check(_lib.tc_debug_flags(ctypes.byref(f), int(bool(clear))), "tc_debug_flags")
    return f.value


def tc_status_string(s: int) -> str:
    return _lib.tc_status_string(s).decode()


# -- convenience wrapper -------------------------------------------------------
class Run:
    """One Taylor-Couette run on the GPU (owns a tc_ctx)."""

    def __init__(self, Nr, Ntheta, Nz, eta, Lz, Re_i, Re_o=0.0, Ra=0.0, Pr=1.0):
        self.ctx = tc_create(Nr, Ntheta, Nz, eta, Lz, Re_i, Re_o, Ra, Pr)
        i = tc_get_info(self.ctx)
        self.Nr, self.Ntheta, self.Nz = i.Nr, i.Ntheta, i.Nz
        self.M, self.K, self.nf = i.M, i.K, i.nfields
        self.shape = (self.nf, self.Nr, self.M + 1, 2 * self.K + 1)
        self.device_bytes = i.device_bytes

    @classmethod
    def from_workload(cls, wl):
        run = cls(wl.Nr, wl.Ntheta, wl.Nz, wl.eta, wl.Lz, wl.Re_i, wl.Re_o, wl.Ra, wl.Pr)
        if wl.dt <= 0:
            tc_set_option(run.ctx, "cfl", wl.cfl)
            tc_set_option(run.ctx, "dt_max", wl.dt_max)
        if getattr(wl, "precision", 0):
            tc_set_option(run.ctx, "precision", wl.precision)
        return run

    def close(self):
        if self.ctx:
            tc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, spec):
        tc_set_state(self.ctx, spec)

    def set_state_regrid(self, spec, eta_src, Lz_src):
        tc_set_state_regrid(self.ctx, spec, eta_src, Lz_src)

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        return tc_get_state(self.ctx, out)

    def get_pressure(self, out=None):
        if out is None:
            out = np.empty(self.shape[1:], dtype=np.complex128)
        return tc_get_pressure(self.ctx, out)

    def init_perturbation(self, psi, amp, tcoef=None, amp_T=0.0):
        tc_init_perturbation(self.ctx, psi, amp, tcoef, amp_T)

    def step(self, nsteps, dt):
        return tc_step(self.ctx, nsteps, dt)

    def get_clock(self):
        return tc_get_clock(self.ctx)

    def set_clock(self, t, dt_prev):
        tc_set_clock(self.ctx, t, dt_prev)

    def diagnostics(self):
        return tc_diagnostics(self.ctx)

    def set_option(self, key, value):
        tc_set_option(self.ctx, key, value)

    def set_stream(self, stream_ptr):
        tc_set_stream(self.ctx, stream_ptr)
