"""Thin ctypes binding of the C ABI in ``include/odegpu.h`` (same names).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``libodegpu.so``.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA; CUDA tensors are passed as device pointers).  A missing or
unloadable library raises ``ODEError``; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# enums of include/odegpu.h
ODE_DUFFING, ODE_KELLER_MIKSIS, ODE_VALVE, ODE_BOUNCE, ODE_DUFFING_LYAPUNOV = 0, 1, 2, 3, 4
ODE_RK4, ODE_RKCK45 = 0, 1
ODE_FP64, ODE_FP32_RHS = 0, 1
ODE_TIMEDOMAIN, ODE_STATE, ODE_PARAM, ODE_ACC, ODE_ALL = 1, 2, 4, 8, 15
ODE_PTR_HOST, ODE_PTR_DEVICE = 0, 1
ODE_TD_KEEP, ODE_TD_T0_TO_T, ODE_TD_SHIFT = 0, 1, 2
(ODE_ST_NONE, ODE_ST_TEND, ODE_ST_EVENT_STOP, ODE_ST_EQUILIBRIUM, ODE_ST_HMIN_NAN,
 ODE_ST_STEP_BUDGET, ODE_ST_TIMEOUT) = range(7)
ODE_OK, ODE_ERR_INVALID_ARG, ODE_ERR_OUT_OF_MEMORY, ODE_ERR_CUDA = 0, -1, -2, -3
ODE_ERR_NOT_READY, ODE_ERR_TIMEOUT, ODE_ERR_UNSUPPORTED = -4, -5, -6

# (n, P, A, E) of each compiled model: state dimension, parameters,
# accessories, events (the hooks of Secs. 6.5-6.8; see include/odegpu.h)
MODEL_DIMS = {ODE_DUFFING: (2, 2, 7, 1), ODE_KELLER_MIKSIS: (2, 13, 4, 1), ODE_VALVE: (3, 5, 5, 2),
              ODE_BOUNCE: (2, 2, 6, 1), ODE_DUFFING_LYAPUNOV: (4, 2, 5, 1)}

# exported symbols, in the order of the header
SYMBOLS = (
    "ode_create", "ode_destroy", "ode_query_dims", "ode_num_systems", "ode_set_tolerances",
    "ode_set_events", "ode_set_model_constants", "ode_set_time_domain_mode", "ode_set_step_budget",
    "ode_set_time_limit", "ode_set_launch", "ode_set_schedule", "ode_linear_set", "ode_random_set", "ode_linear_get", "ode_random_get",
    "ode_solve", "ode_run_periods", "ode_autotune", "ode_synchronize", "ode_get_status", "ode_reset_counters",
    "ode_last_error", "ode_km_coefficients", "ode_cluster_order", "ode_kernel_info", "ode_probe_fma_peak",
    "ode_probe_call_cost", "ode_run_periods_noalloc",
    "ode_server_create", "ode_server_add_model", "ode_server_submit", "ode_server_progress",
    "ode_server_poll", "ode_server_result", "ode_server_stats", "ode_server_destroy", "ode_server_last_error",
)


class NoAllocSettings(ctypes.Structure):
    """Mirror of ``ode_noalloc_settings``."""

    _fields_ = [
        ("model", ctypes.c_int), ("scheme", ctypes.c_int), ("prec", ctypes.c_int),
        ("rtol", ctypes.c_double * 4), ("atol", ctypes.c_double * 4),
        ("h_max", ctypes.c_double), ("h_min", ctypes.c_double), ("grow_limit", ctypes.c_double),
        ("shrink_limit", ctypes.c_double), ("events_enabled", ctypes.c_int),
        ("direction", ctypes.c_int * 2), ("tolerance", ctypes.c_double * 2),
        ("stop_count", ctypes.c_int * 2), ("max_steps_in_zone", ctypes.c_int),
        ("time_domain_mode", ctypes.c_int), ("max_steps_per_slice", ctypes.c_longlong),
        ("time_limit_s", ctypes.c_double), ("model_constants", ctypes.c_double * 8),
    ]


class ODEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("odegpu error %d: %s" % (code, msg))
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_longlong)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libodegpu.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ODEError(ODE_ERR_UNSUPPORTED, "libodegpu.so is not built (run build())")
    L = ctypes.CDLL(_build.LIB)
    i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "ode_create": [ctypes.POINTER(_vp), i, i, i, i, i],
        "ode_destroy": [_vp],
        "ode_query_dims": [_vp, _ip, _ip, _ip, _ip],
        "ode_num_systems": [_vp, _ip],
        "ode_set_tolerances": [_vp, _dp, _dp, d, d, d, d],
        "ode_set_events": [_vp, i, _ip, _dp, _ip, i],
        "ode_set_model_constants": [_vp, _dp, i],
        "ode_set_time_domain_mode": [_vp, i],
        "ode_set_step_budget": [_vp, ll],
        "ode_set_time_limit": [_vp, d],
        "ode_set_launch": [_vp, i, i],
        "ode_linear_set": [_vp, i, i, i, i, _vp, _vp, _vp, _vp, i, i, _vp],
        "ode_random_set": [_vp, _vp, _vp, i, i, _vp, _vp, _vp, _vp, i, i, _vp],
        "ode_linear_get": [_vp, i, i, i, i, _vp, _vp, _vp, _vp, i, i, _vp],
        "ode_random_get": [_vp, _vp, _vp, i, i, _vp, _vp, _vp, _vp, i, i, _vp],
        "ode_solve": [_vp, d, _vp],
        "ode_run_periods": [_vp, d, i, i, _vp, i, _vp],
        "ode_autotune": [_vp, d, i, _vp, _ip, _ip, _ip, _ip, _ip, _dp],
        "ode_set_schedule": [_vp, i, i, i],
        "ode_synchronize": [_vp],
        "ode_get_status": [_vp, _vp, _vp, _vp, _vp, i, _vp],
        "ode_reset_counters": [_vp, _vp],
        "ode_last_error": [_vp],
        "ode_km_coefficients": [d] * 13 + [_dp],
        "ode_cluster_order": [_dp, i, i, _ip],
        "ode_kernel_info": [i, i, i, i, i, i, _ip, _ip, _ip],
        "ode_probe_fma_peak": [i, _dp, _dp],
        "ode_probe_call_cost": [i, _dp, _dp, _dp],
        "ode_run_periods_noalloc": [ctypes.POINTER(NoAllocSettings), i, i, d, i, i, _vp, _vp, _vp, _vp,
                                    _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_char_p)],
    }
    sp = ctypes.POINTER(NoAllocSettings)
    sig.update({
        "ode_server_create": [ctypes.POINTER(_vp), i, ll, i],
        "ode_server_add_model": [_vp, sp, d, i],
        "ode_server_submit": [_vp, i, i, i, _dp, _dp, _dp, ctypes.POINTER(ll)],
        "ode_server_progress": [_vp, _ip, _ip],
        "ode_server_poll": [_vp, ll, _ip],
        "ode_server_result": [_vp, ll, _dp, _dp, _dp, _ip, _lp, _dp],
        "ode_server_stats": [_vp, i, _lp],
        "ode_server_destroy": [_vp],
        "ode_server_last_error": [_vp],
    })
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name.endswith("last_error") else ctypes.c_int
    _lib = L
    return L


def ode_last_error(s=None) -> str:
    msg = load().ode_last_error(s)
    return msg.decode() if msg else ""


def _check(rc, s=None):
    if rc != ODE_OK:
        raise ODEError(rc, ode_last_error(s))
    return rc


# ---- array marshalling ---------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arr(x, dtype):
    """(pointer as int or None, ptr_kind or None) for numpy / torch arrays."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = torch.float64 if dtype == np.float64 else (torch.int32 if dtype == np.int32 else torch.int64)
        if x.dtype != want or not x.is_contiguous():
            raise ODEError(ODE_ERR_INVALID_ARG, "tensor must be contiguous %s" % want)
        return x.data_ptr(), (ODE_PTR_DEVICE if x.is_cuda else ODE_PTR_HOST)
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise ODEError(ODE_ERR_INVALID_ARG, "array must be a C-contiguous numpy %s array" % np.dtype(dtype))
    return x.ctypes.data, ODE_PTR_HOST


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ODEError(ODE_ERR_INVALID_ARG, "mixing host and device arrays in one call")
    return ks.pop() if ks else ODE_PTR_HOST


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ---- C ABI, same names -----------------------------------------------------------
def ode_create(model, scheme, prec, n_systems, device=0):
    h = _vp()
    _check(load().ode_create(ctypes.byref(h), model, scheme, prec, n_systems, device))
    return h


def ode_destroy(s):
    return _check(load().ode_destroy(s))


def ode_query_dims(s):
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().ode_query_dims(s, *[ctypes.byref(x) for x in v]), s)
    return tuple(x.value for x in v)  # (n, P, E, A)


def ode_num_systems(s):
    v = ctypes.c_int()
    _check(load().ode_num_systems(s, ctypes.byref(v)), s)
    return v.value


def ode_set_tolerances(s, rtol, atol, h_max, h_min, grow_limit, shrink_limit):
    r = np.ascontiguousarray(rtol, dtype=np.float64)
    a = np.ascontiguousarray(atol, dtype=np.float64)
    return _check(load().ode_set_tolerances(s, r.ctypes.data_as(_dp), a.ctypes.data_as(_dp),
                                            h_max, h_min, grow_limit, shrink_limit), s)


def ode_set_events(s, enabled, direction=None, tolerance=None, stop_count=None, max_steps_in_zone=0):
    d = None if direction is None else np.ascontiguousarray(direction, dtype=np.int32)
    t = None if tolerance is None else np.ascontiguousarray(tolerance, dtype=np.float64)
    c = None if stop_count is None else np.ascontiguousarray(stop_count, dtype=np.int32)
    return _check(load().ode_set_events(
        s, int(enabled), None if d is None else d.ctypes.data_as(_ip),
        None if t is None else t.ctypes.data_as(_dp), None if c is None else c.ctypes.data_as(_ip),
        int(max_steps_in_zone)), s)


def ode_set_model_constants(s, c):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _check(load().ode_set_model_constants(s, c.ctypes.data_as(_dp), c.size), s)


def ode_set_time_domain_mode(s, mode):
    return _check(load().ode_set_time_domain_mode(s, mode), s)


def ode_set_step_budget(s, max_steps):
    return _check(load().ode_set_step_budget(s, int(max_steps)), s)


def ode_set_time_limit(s, seconds):
    return _check(load().ode_set_time_limit(s, float(seconds)), s)


def ode_set_launch(s, block_size=0, persistent=0):
    return _check(load().ode_set_launch(s, int(block_size), int(persistent)), s)


def _copy(fn, s, a0, a1, pool_size, count, td, y, p, acc, copy_mode, stream, idx=False):
    ptrs = [_arr(x, np.float64) for x in (td, y, p, acc)]
    if idx:
        i0, k0 = _arr(a0, np.int32)
        i1, k1 = _arr(a1, np.int32)
        kind = _kind(k0, k1, *[k for _, k in ptrs])
        a0, a1 = i0, i1
    else:
        kind = _kind(*[k for _, k in ptrs])
    return _check(fn(s, a0, a1, pool_size, count, *[pp for pp, _ in ptrs], copy_mode, kind,
                     _stream(stream)), s)


def ode_linear_set(s, start_obj, start_pool, pool_size, count, td=None, y=None, p=None, acc=None,
                   copy_mode=ODE_ALL, stream=None):
    return _copy(load().ode_linear_set, s, start_obj, start_pool, pool_size, count, td, y, p, acc,
                 copy_mode, stream)


def ode_linear_get(s, start_obj, start_pool, pool_size, count, td=None, y=None, p=None, acc=None,
                   copy_mode=ODE_ALL, stream=None):
    return _copy(load().ode_linear_get, s, start_obj, start_pool, pool_size, count, td, y, p, acc,
                 copy_mode, stream)


def ode_random_set(s, idx_obj, idx_pool, pool_size, count, td=None, y=None, p=None, acc=None,
                   copy_mode=ODE_ALL, stream=None):
    return _copy(load().ode_random_set, s, idx_obj, idx_pool, pool_size, count, td, y, p, acc,
                 copy_mode, stream, idx=True)


def ode_random_get(s, idx_obj, idx_pool, pool_size, count, td=None, y=None, p=None, acc=None,
                   copy_mode=ODE_ALL, stream=None):
    return _copy(load().ode_random_get, s, idx_obj, idx_pool, pool_size, count, td, y, p, acc,
                 copy_mode, stream, idx=True)


def ode_solve(s, h0, stream=None):
    return _check(load().ode_solve(s, h0, _stream(stream)), s)


def ode_run_periods(s, h0, n_transient, n_record, records=None, stream=None):
    ptr, kind = _arr(records, np.float64)
    return _check(load().ode_run_periods(s, h0, n_transient, n_record, ptr,
                                         ODE_PTR_HOST if kind is None else kind, _stream(stream)), s)


def ode_autotune(s, h0, n_slices, stream=None, full=False):
    """Returns (block, persistent, trial_ms[4][6]); with full=True a dict that
    adds systems_per_thread, slices_per_launch, warp_sync, the schedule
    trials of the fastest shape [1 slice per launch, half, all, all
    warp-synchronous] and the warp-synchronous trial of every form at its
    fastest block (warp_sync_ms[4])."""
    b, pr, spt, spl, ws = (ctypes.c_int() for _ in range(5))
    ms = np.zeros(32)
    _check(load().ode_autotune(s, h0, n_slices, _stream(stream), ctypes.byref(b), ctypes.byref(pr),
                               ctypes.byref(spt), ctypes.byref(spl), ctypes.byref(ws),
                               ms.ctypes.data_as(_dp)), s)
    if full:
        return dict(block=b.value, persistent=pr.value, systems_per_thread=spt.value,
                    slices_per_launch=spl.value, warp_sync=ws.value, trial_ms=ms[:24].reshape(4, 6),
                    split_ms=ms[24:28], warp_sync_ms=ms[28:32])
    return b.value, pr.value, ms[:24].reshape(4, 6)


def ode_set_schedule(s, systems_per_thread=1, slices_per_launch=0, warp_sync=0):
    return _check(load().ode_set_schedule(s, int(systems_per_thread), int(slices_per_launch), int(warp_sync)), s)


def ode_synchronize(s):
    return _check(load().ode_synchronize(s), s)


def ode_get_status(s, status=None, accepted=None, rejected=None, event_counts=None, stream=None):
    a = _arr(status, np.int32)
    b = _arr(accepted, np.int64)
    c = _arr(rejected, np.int64)
    d = _arr(event_counts, np.int32)
    kind = _kind(a[1], b[1], c[1], d[1])
    return _check(load().ode_get_status(s, a[0], b[0], c[0], d[0], kind, _stream(stream)), s)


def ode_reset_counters(s, stream=None):
    return _check(load().ode_reset_counters(s, _stream(stream)), s)


def ode_km_coefficients(PA1, PA2, omega1, omega2, theta, RE, Pinf, pV, sigma, mu, rho, cL, gamma):
    C = np.zeros(13)
    _check(load().ode_km_coefficients(PA1, PA2, omega1, omega2, theta, RE, Pinf, pV, sigma, mu, rho,
                                      cL, gamma, C.ctypes.data_as(_dp)))
    return C


def ode_cluster_order(keys):
    """Permutation of the N systems along a Z-order curve of `keys` (K x N):
    slot i should hold system perm[i]."""
    k = np.ascontiguousarray(np.atleast_2d(np.asarray(keys, dtype=np.float64)))
    perm = np.zeros(k.shape[1], dtype=np.int32)
    _check(load().ode_cluster_order(k.ctypes.data_as(_dp), k.shape[0], k.shape[1], perm.ctypes.data_as(_ip)))
    return perm


def ode_kernel_info(model, scheme, prec, persistent=0, block_size=0, device=0):
    r, l, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().ode_kernel_info(model, scheme, prec, persistent, block_size, device, ctypes.byref(r),
                                  ctypes.byref(l), ctypes.byref(b)))
    return dict(regs=r.value, local_bytes=l.value, blocks_per_sm=b.value)


def ode_probe_call_cost(device=0):
    """(cos, pow, sqrt) cost in DFMA equivalents."""
    c, p, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().ode_probe_call_cost(device, ctypes.byref(c), ctypes.byref(p), ctypes.byref(q)))
    return c.value, p.value, q.value


def ode_probe_fma_peak(device=0):
    d, f = ctypes.c_double(), ctypes.c_double()
    _check(load().ode_probe_fma_peak(device, ctypes.byref(d), ctypes.byref(f)))
    return d.value, f.value


def ode_run_periods_noalloc(settings, n_systems, device, h0, n_transient, n_record, td, y, p, acc,
                            records=None, status=None, accepted=None, stream=None):
    """Integration on caller-owned device arrays with no device allocation
    (see include/odegpu.h).  Arrays must be contiguous CUDA tensors on
    `device` holding at least the elements the call reads or writes (td 2N,
    y nN, p PN, acc AN, records n_record (A+n+1) N, status and accepted N),
    else ODEError(ODE_ERR_INVALID_ARG) is raised before the library is
    called; raw device pointers (ints) are passed unchecked."""
    dims = MODEL_DIMS.get(settings.model)
    N = int(n_systems)
    if dims is not None and N >= 1:
        n, P, A, E = dims
        need = dict(td=2 * N, y=n * N, p=P * N, acc=A * N, records=max(0, n_record) * (A + n + 1) * N,
                    status=N, accepted=N)
    else:
        need = {}  # the library rejects the model or size itself

    def dev(name, x, dtype):
        if x is None or isinstance(x, int):
            return x
        ptr, kind = _arr(x, dtype)  # checks dtype and contiguity
        if kind != ODE_PTR_DEVICE:
            raise ODEError(ODE_ERR_INVALID_ARG, "ode_run_periods_noalloc takes device arrays only")
        if x.device.index != device:
            raise ODEError(ODE_ERR_INVALID_ARG, "%s is on cuda:%s, not on device %d" % (name, x.device.index, device))
        if name in need and x.numel() < need[name]:
            raise ODEError(ODE_ERR_INVALID_ARG, "%s holds %d elements, the call needs %d"
                           % (name, x.numel(), need[name]))
        return ptr
    msg = ctypes.c_char_p()
    rc = load().ode_run_periods_noalloc(
        ctypes.byref(settings), n_systems, device, h0, n_transient, n_record, dev("td", td, np.float64),
        dev("y", y, np.float64), dev("p", p, np.float64), dev("acc", acc, np.float64),
        dev("records", records, np.float64), dev("status", status, np.int32),
        dev("accepted", accepted, np.int64), _stream(stream), ctypes.byref(msg))
    if rc != ODE_OK:
        raise ODEError(rc, msg.value.decode() if msg.value else "")
    return rc


# ---- serving -------------------------------------------------------------------
def _scheck(rc, s):
    if rc != ODE_OK:
        msg = load().ode_server_last_error(s) if s else b""
        raise ODEError(rc, msg.decode() if msg else "server call failed")
    return rc


def ode_server_create(device, hbm_budget_bytes, slice_periods):
    h = _vp()
    _scheck(load().ode_server_create(ctypes.byref(h), device, int(hbm_budget_bytes), int(slice_periods)), None)
    return h


def ode_server_add_model(s, settings, h0, capacity):
    return _scheck(load().ode_server_add_model(s, ctypes.byref(settings), h0, int(capacity)), s)


def ode_server_submit(s, model, n_periods, td, y0, p):
    td = np.ascontiguousarray(td, dtype=np.float64)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    t = ctypes.c_longlong()
    _scheck(load().ode_server_submit(s, model, td.shape[1], int(n_periods), td.ctypes.data_as(_dp),
                                     y0.ctypes.data_as(_dp), p.ctypes.data_as(_dp), ctypes.byref(t)), s)
    return t.value


def ode_server_progress(s):
    r, w = ctypes.c_int(), ctypes.c_int()
    _scheck(load().ode_server_progress(s, ctypes.byref(r), ctypes.byref(w)), s)
    return r.value, w.value


def ode_server_poll(s, ticket):
    st = ctypes.c_int()
    _scheck(load().ode_server_poll(s, ticket, ctypes.byref(st)), s)
    return st.value


def ode_server_result(s, ticket, n, n_sys, n_acc):
    td, y, acc = np.zeros((2, n)), np.zeros((n_sys, n)), np.zeros((n_acc, n))
    status = np.zeros(n, dtype=np.int32)
    accepted = np.zeros(n, dtype=np.int64)
    lat = ctypes.c_double()
    _scheck(load().ode_server_result(s, ticket, td.ctypes.data_as(_dp), y.ctypes.data_as(_dp),
                                     acc.ctypes.data_as(_dp), status.ctypes.data_as(_ip),
                                     accepted.ctypes.data_as(_lp), ctypes.byref(lat)), s)
    return dict(td=td, y=y, acc=acc, status=status, nacc=accepted, latency=lat.value)


def ode_server_stats(s, model):
    out = np.zeros(8, dtype=np.int64)
    _scheck(load().ode_server_stats(s, int(model), out.ctypes.data_as(_lp)), s)
    keys = ("launches", "stops", "yielded", "snapshots", "published", "finished", "flags", "unfinished")
    return dict(zip(keys, (int(x) for x in out)))


def ode_server_destroy(s):
    return _scheck(load().ode_server_destroy(s), None)


def ode_server_last_error(s):
    m = load().ode_server_last_error(s)
    return m.decode() if m else ""
