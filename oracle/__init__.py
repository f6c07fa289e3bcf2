"""CPU oracle for the integration method of arXiv:1810.03931 -- TEST INFRASTRUCTURE.

This package is a plain, slow FP64 restatement of the method in C
(``oracle.c``), loaded through ctypes.  Only ``tests/``, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
product library never does, and the two share no code.

Every per-system array is structure-of-arrays, ``a[component, system]`` as the
problem pool of Sec. 6.1 of the paper prescribes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DUFFING, KELLER_MIKSIS, VALVE, BOUNCE, DUFFING_LYAPUNOV = 0, 1, 2, 3, 4
RK4, RKCK45 = 0, 1
TD_KEEP, TD_T0_TO_T, TD_SHIFT = 0, 1, 2
ST_NONE, ST_TEND, ST_EVENT_STOP, ST_EQUILIBRIUM, ST_HMIN_NAN, ST_STEP_BUDGET = range(6)

MAXN, MAXP, MAXA, MAXE = 4, 16, 8, 2


class Config(ctypes.Structure):
    """Mirror of ``orc_config`` (ODE properties Sec. 6.5, event properties
    Sec. 6.6, solver configuration Sec. 6.4)."""

    _fields_ = [
        ("model", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("events_on", ctypes.c_int),
        ("td_mode", ctypes.c_int),
        ("h0", ctypes.c_double),
        ("rtol", ctypes.c_double * MAXN),
        ("atol", ctypes.c_double * MAXN),
        ("hmax", ctypes.c_double),
        ("hmin", ctypes.c_double),
        ("grow", ctypes.c_double),
        ("shrink", ctypes.c_double),
        ("evt_dir", ctypes.c_int * MAXE),
        ("evt_tol", ctypes.c_double * MAXE),
        ("evt_stop", ctypes.c_int * MAXE),
        ("max_eq", ctypes.c_int),
        ("max_steps", ctypes.c_longlong),
        ("mc", ctypes.c_double * 8),
    ]


class _Trace(ctypes.Structure):
    _fields_ = [
        ("cap", ctypes.c_int),
        ("n_points", ctypes.c_int),
        ("t", ctypes.POINTER(ctypes.c_double)),
        ("y", ctypes.POINTER(ctypes.c_double)),
        ("ev_cap", ctypes.c_int),
        ("n_events", ctypes.c_int),
        ("ev_index", ctypes.POINTER(ctypes.c_int)),
        ("ev_t", ctypes.POINTER(ctypes.c_double)),
        ("ev_y", ctypes.POINTER(ctypes.c_double)),
        ("ev_y_after", ctypes.POINTER(ctypes.c_double)),
        ("trial_cap", ctypes.c_int),
        ("n_trials", ctypes.c_int),
        ("trial_t", ctypes.POINTER(ctypes.c_double)),
        ("trial_h", ctypes.POINTER(ctypes.c_double)),
        ("trial_y", ctypes.POINTER(ctypes.c_double)),
        ("trial_ynew", ctypes.POINTER(ctypes.c_double)),
        ("trial_e", ctypes.POINTER(ctypes.c_double)),
        ("trial_ok", ctypes.POINTER(ctypes.c_int)),
        ("trial_hnext", ctypes.POINTER(ctypes.c_double)),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, FP64,
    no FMA contraction).  Returns the library path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.run(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                 "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"],
                check=True,
            )
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_longlong)
        L.orc_dims.argtypes = [ctypes.c_int, ip, ip, ip, ip]
        L.orc_run.argtypes = [ctypes.POINTER(Config), ctypes.c_int, dp, dp, dp, dp, ip, ip, lp, lp,
                              ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
        L.orc_trace_slice.argtypes = [ctypes.POINTER(Config), dp, dp, dp, dp, ip, lp, lp,
                                      ctypes.POINTER(_Trace)]
        L.orc_single_step.argtypes = [ctypes.POINTER(Config), ctypes.c_double, dp, dp,
                                      ctypes.c_double, dp, dp]
        L.orc_rhs.argtypes = [ctypes.POINTER(Config), ctypes.c_double, dp, dp, dp]
        L.orc_ck_tableau.argtypes = [dp, dp, dp, dp]
        L.orc_rk4_tableau.argtypes = [dp, dp, dp]
        L.orc_km_coefficients.argtypes = [ctypes.c_double] * 13 + [dp]
        _lib = L
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of the
    oracle (tests compile deliberately broken copies to show that the pins
    catch them)."""

    def __init__(self, path):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        self.saved = lib()
        L = ctypes.CDLL(self.path)
        for name in ("orc_dims", "orc_run", "orc_trace_slice", "orc_single_step", "orc_rhs",
                     "orc_ck_tableau", "orc_rk4_tableau", "orc_km_coefficients"):
            getattr(L, name).argtypes = getattr(self.saved, name).argtypes
        _lib = L
        return L

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def build_variant(source_text, out_path):
    """Compile a modified oracle source into `out_path` (tests only)."""
    src = out_path[:-3] + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
                    "-D_GNU_SOURCE", "-o", out_path, src, "-lm", "-lpthread"], check=True)
    return out_path


def source():
    with open(_SRC) as f:
        return f.read()


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if a is not None else None


def dims(model: int):
    """(n, P, A, E): state dimension, parameters, accessories, events."""
    n, P, A, E = (ctypes.c_int() for _ in range(4))
    if lib().orc_dims(model, ctypes.byref(n), ctypes.byref(P), ctypes.byref(A), ctypes.byref(E)):
        raise ValueError("unknown model %r" % model)
    return n.value, P.value, A.value, E.value


DEFAULT_MC = {
    DUFFING: (-1.0, 1.0, 1.0),   # delta, c3, omega: x'' + k x' + x + x^3 = B cos t
    DUFFING_LYAPUNOV: (-1.0, 1.0, 1.0),
}


def make_config(model, scheme, h0, rtol=1e-10, atol=1e-10, hmax=1e6, hmin=1e-12, grow=5.0,
                shrink=0.1, events_on=False, evt_dir=(-1, -1), evt_tol=(1e-6, 1e-6),
                evt_stop=(0, 0), max_eq=0, max_steps=10**12, mc=None, td_mode=TD_KEEP) -> Config:
    """Build an oracle configuration.  Scalars rtol/atol apply to every
    component; defaults of hmax, hmin, grow and shrink follow Sec. 6.5."""
    c = Config()
    c.model, c.scheme, c.events_on, c.td_mode = model, scheme, int(bool(events_on)), td_mode
    c.h0 = h0
    rt = np.broadcast_to(np.asarray(rtol, dtype=np.float64), (MAXN,)) if np.ndim(rtol) == 0 else rtol
    at = np.broadcast_to(np.asarray(atol, dtype=np.float64), (MAXN,)) if np.ndim(atol) == 0 else atol
    for i in range(MAXN):
        c.rtol[i] = float(rt[i]) if i < len(rt) else float(rt[-1])
        c.atol[i] = float(at[i]) if i < len(at) else float(at[-1])
    c.hmax, c.hmin, c.grow, c.shrink = hmax, hmin, grow, shrink
    for j in range(MAXE):
        c.evt_dir[j] = int(evt_dir[j]) if j < len(evt_dir) else -1
        c.evt_tol[j] = float(evt_tol[j]) if j < len(evt_tol) else 1e-6
        c.evt_stop[j] = int(evt_stop[j]) if j < len(evt_stop) else 0
    c.max_eq = max_eq
    c.max_steps = max_steps
    if mc is None:
        mc = DEFAULT_MC.get(model, ())
    for i in range(8):
        c.mc[i] = float(mc[i]) if i < len(mc) else 0.0
    return c


def run(cfg: Config, td, y, p, acc=None, n_slices=1, n_skip=0, record=False, nthreads=1):
    """Integrate every system over ``n_slices`` consecutive slices.

    td: (2, N); y: (n, N); p: (P, N); acc: (A, N) or None (zeros).  Inputs are
    copied.  Returns a dict with td, y, acc, status, ecnt, nacc, nrej and, if
    ``record``, records of shape (n_slices - n_skip, A + n + 1, N).
    """
    n, P, A, E = dims(cfg.model)
    td = np.array(td, dtype=np.float64, order="C", copy=True).reshape(2, -1)
    N = td.shape[1]
    y = np.array(y, dtype=np.float64, order="C", copy=True).reshape(n, N)
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(P, N))
    acc = np.zeros((A, N)) if acc is None else np.array(acc, dtype=np.float64, order="C", copy=True)
    status = np.zeros(N, dtype=np.int32)
    ecnt = np.zeros((E, N), dtype=np.int32)
    nacc = np.zeros(N, dtype=np.int64)
    nrej = np.zeros(N, dtype=np.int64)
    R = A + n + 1
    nrec = max(n_slices - n_skip, 0)
    records = np.zeros((nrec, R, N)) if record and nrec > 0 else None
    rc = lib().orc_run(ctypes.byref(cfg), N, _dp(td), _dp(y), _dp(p), _dp(acc), _ip(status), _ip(ecnt),
                       _lp(nacc), _lp(nrej), n_slices, n_skip, _dp(records), nthreads)
    if rc:
        raise ValueError("orc_run failed (%d)" % rc)
    out = dict(td=td, y=y, acc=acc, status=status, ecnt=ecnt, nacc=nacc, nrej=nrej)
    if records is not None:
        out["records"] = records
    return out


def trace_slice(cfg: Config, td, y, p, acc=None, cap=1_000_000, ev_cap=100_000, trial_cap=0):
    """One slice of ONE system, returning every accepted point and event, and
    (trial_cap > 0) the first trial_cap trial steps of the adaptive scheme:
    start time, step size, start state, result, error estimate, outcome
    (1 accepted, 0 rejected, -1 non-finite) and the step chosen next."""
    n, P, A, E = dims(cfg.model)
    td = np.array(td, dtype=np.float64).reshape(2).copy()
    y = np.array(y, dtype=np.float64).reshape(n).copy()
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(P))
    acc = np.zeros(A) if acc is None else np.array(acc, dtype=np.float64).copy()
    ecnt = np.zeros(MAXE, dtype=np.int32)
    nacc = np.zeros(1, dtype=np.int64)
    nrej = np.zeros(1, dtype=np.int64)
    tbuf = np.zeros(cap)
    ybuf = np.zeros((cap, MAXN))
    ev_index = np.zeros(ev_cap, dtype=np.int32)
    ev_t = np.zeros(ev_cap)
    ev_y = np.zeros((ev_cap, MAXN))
    ev_y_after = np.zeros((ev_cap, MAXN))
    tc = max(0, int(trial_cap))
    tt, th, thn = np.zeros(max(tc, 1)), np.zeros(max(tc, 1)), np.zeros(max(tc, 1))
    ty, tyn, te = (np.zeros((max(tc, 1), MAXN)) for _ in range(3))
    tok = np.zeros(max(tc, 1), dtype=np.int32)
    tr = _Trace(cap, 0, _dp(tbuf), _dp(ybuf), ev_cap, 0, _ip(ev_index), _dp(ev_t), _dp(ev_y),
                _dp(ev_y_after), tc, 0, _dp(tt), _dp(th), _dp(ty), _dp(tyn), _dp(te), _ip(tok), _dp(thn))
    st = lib().orc_trace_slice(ctypes.byref(cfg), _dp(td), _dp(y), _dp(p), _dp(acc), _ip(ecnt),
                               _lp(nacc), _lp(nrej), ctypes.byref(tr))
    k, m = tr.n_points, tr.n_events
    return dict(status=st, td=td, y=y, acc=acc, ecnt=ecnt[:E].copy(), nacc=int(nacc[0]),
                nrej=int(nrej[0]), t=tbuf[:k].copy(), ys=ybuf[:k, :n].copy(),
                ev_index=ev_index[:m].copy(), ev_t=ev_t[:m].copy(), ev_y=ev_y[:m, :n].copy(),
                ev_y_after=ev_y_after[:m, :n].copy(),
                trials=dict(t=tt[:tr.n_trials].copy(), h=th[:tr.n_trials].copy(),
                            y=ty[:tr.n_trials, :n].copy(), ynew=tyn[:tr.n_trials, :n].copy(),
                            e=te[:tr.n_trials, :n].copy(), ok=tok[:tr.n_trials].copy(),
                            hnext=thn[:tr.n_trials].copy()))


def single_step(cfg: Config, t, y, p, h):
    """One Runge-Kutta step of size h; returns (y_new, error_estimate)."""
    n, P, A, E = dims(cfg.model)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(n))
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(P))
    ynew = np.zeros(n)
    err = np.zeros(n)
    lib().orc_single_step(ctypes.byref(cfg), t, _dp(y), _dp(p), h, _dp(ynew), _dp(err))
    return ynew, err


def rhs(cfg: Config, t, y, p):
    n, P, A, E = dims(cfg.model)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(n))
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(P))
    f = np.zeros(n)
    lib().orc_rhs(ctypes.byref(cfg), t, _dp(y), _dp(p), _dp(f))
    return f


def ck_tableau():
    """(c[6], a[6,6], b5[6], b4[6]) of the oracle's Cash-Karp pair."""
    c, a, b5, b4 = np.zeros(6), np.zeros((6, 6)), np.zeros(6), np.zeros(6)
    lib().orc_ck_tableau(_dp(c), _dp(a), _dp(b5), _dp(b4))
    return c, a, b5, b4


def rk4_tableau():
    c, a, b = np.zeros(4), np.zeros((4, 4)), np.zeros(4)
    lib().orc_rk4_tableau(_dp(c), _dp(a), _dp(b))
    return c, a, b


# Physical constants of the Keller-Miksis workload (SI units).
KM_WATER = dict(Pinf=1.0e5, pV=3166.8, sigma=0.072, mu=8.9e-4, rho=997.0, cL=1497.0, gamma=1.4,
                RE=10e-6)


def km_coefficients(PA1, omega1, PA2=0.0, omega2=None, theta=0.0, **phys):
    """C0..C12 of Eqs. (16)-(28) for arrays of (PA1 [Pa], omega1 [rad/s]).
    Returns an array of shape (13, N)."""
    ph = dict(KM_WATER)
    ph.update(phys)
    PA1 = np.atleast_1d(np.asarray(PA1, dtype=np.float64))
    omega1 = np.broadcast_to(np.asarray(omega1, dtype=np.float64), PA1.shape)
    PA2 = np.broadcast_to(np.asarray(PA2, dtype=np.float64), PA1.shape)
    omega2 = omega1 if omega2 is None else np.broadcast_to(np.asarray(omega2, dtype=np.float64), PA1.shape)
    theta = np.broadcast_to(np.asarray(theta, dtype=np.float64), PA1.shape)
    out = np.zeros((13, PA1.size))
    C = np.zeros(13)
    for i in range(PA1.size):
        lib().orc_km_coefficients(PA1.flat[i], PA2.flat[i], omega1.flat[i], omega2.flat[i], theta.flat[i],
                                  ph["RE"], ph["Pinf"], ph["pV"], ph["sigma"], ph["mu"], ph["rho"],
                                  ph["cL"], ph["gamma"], _dp(C))
        out[:, i] = C
    return out


def run_workload(w, nthreads=8, record=True, n_transient=None, n_record=None, **cfg_over):
    """Run a seeded sweep description (the ``workloads`` dictionaries) through
    the oracle: its settings, time domains, initial conditions and parameters
    (Keller-Miksis coefficients from this module's own Eqs. 16-28 code).
    ``cfg_over`` overrides settings (e.g. rtol, atol)."""
    n_tr = w["n_transient"] if n_transient is None else n_transient
    n_rec = w["n_record"] if n_record is None else n_record
    ww = dict(w)
    ww.update(cfg_over)
    cfg = make_config(ww["model"], ww["scheme"], ww["h0"], rtol=ww["rtol"], atol=ww["atol"], hmax=ww["hmax"],
                      hmin=ww["hmin"], grow=ww["grow"], shrink=ww["shrink"], events_on=ww["events_on"],
                      evt_dir=ww["evt_dir"], evt_tol=ww["evt_tol"], evt_stop=ww["evt_stop"], max_eq=ww["max_eq"],
                      mc=ww["mc"] or None, td_mode=ww["td_mode"])
    if w["model"] == KELLER_MIKSIS:
        N = w["N"]
        p = km_coefficients(w["PA"], w["omega"], PA2=w.get("PA2", np.zeros(N)),
                            omega2=w.get("omega2", w["omega"]), theta=0.0, **w["phys"])
    else:
        p = w["p"]
    return run(cfg, w["td"], w["y0"], p, None, n_slices=n_tr + n_rec, n_skip=n_tr, record=record,
               nthreads=nthreads)
