"""Seeded synthetic inputs shaped like the paper's test cases.

This module only lays out parameter grids, initial conditions, time domains
and solver settings (and the random request stream of the serving mix).  It
holds none of the integration method's arithmetic, so both the CUDA path and
the CPU oracle can take their inputs from it.  Keller-Miksis cases give the
PHYSICAL parameters (pressure amplitude, frequency); each side computes its
own coefficients C0..C12 from them.

Workloads (the paper's experiments, Sec. 7, at the sizes of the benchmark):
  duffing_rk4    Duffing, RK4 dt = 2 pi / 1000, N = 1024, k in [0.2, 0.3],
                 B = 0.3, y0 = (-0.5, 0.1), 64 transient + 32 recorded periods
  duffing_rkck   Duffing, RKCK45 rtol = atol = 1e-10, h0 = 1e-2, 512 x 256
                 grid of k in [0.2, 0.3] (fastest) x B in [0.3, 0.5], event
                 y2 = 0 downwards (local maxima) located to 1e-12,
                 1024 transient + 64 recorded periods
  keller_miksis  Keller-Miksis single frequency, 512 x 512 grid of
                 pA in [0, 2] bar (linear) x f in [20, 1000] kHz (log,
                 fastest), y0 = (1, 0), slices of one acoustic period,
                 RKCK45 rtol 1e-10, 1024 + 64 periods
  valve          pressure relief valve, q in [0.2, 10] over 2^16 systems,
                 events (y2 max, stop 1) and (y1 impact), equilibrium 50,
                 y0 = (0.2, 0, delta), slices of up to 1e3 time units that
                 stop at the next maximum, RKCK45 rtol 1e-9, 1024 + 64
  duffing_lyapunov  Duffing with its polar linearisation (largest Lyapunov
                 exponent, Sec. 7.1.3): k in [0.2, 0.3] over 61440 systems,
                 B = 0.3, y0 = (-0.5, 0.1, 1, 0), RKCK45 rtol = atol = 1e-9,
                 slices of one forcing period, 1024 + 64 periods
  serving_mix    Poisson stream of sweep requests over the three models
"""
from __future__ import annotations

import math

import numpy as np

DUFFING, KELLER_MIKSIS, VALVE, BOUNCE, DUFFING_LYAPUNOV = 0, 1, 2, 3, 4
RK4, RKCK45 = 0, 1
TD_KEEP, TD_T0_TO_T, TD_SHIFT = 0, 1, 2

KM_PHYS = dict(Pinf=1.0e5, pV=3166.8, sigma=0.072, mu=8.9e-4, rho=997.0, cL=1497.0, gamma=1.4,
               RE=10e-6)
VALVE_FIXED = dict(kappa=1.25, delta=10.0, beta=20.0, r=0.8)
SEED = 1810003931


def _base(**kw):
    d = dict(rtol=1e-10, atol=1e-10, hmax=1e6, hmin=1e-12, grow=5.0, shrink=0.1, events_on=False,
             evt_dir=(-1, -1), evt_tol=(1e-6, 1e-6), evt_stop=(0, 0), max_eq=0, td_mode=TD_KEEP,
             mc=(), n_transient=0, n_record=1)
    d.update(kw)
    return d


def duffing_rk4(N=1024, n_transient=64, n_record=32):
    k = np.linspace(0.2, 0.3, N)
    B = np.full(N, 0.3)
    return _base(name="duffing_rk4_%d" % N, model=DUFFING, scheme=RK4, N=N, h0=2 * math.pi / 1000,
                 td=np.vstack([np.zeros(N), np.full(N, 2 * math.pi)]),
                 y0=np.vstack([np.full(N, -0.5), np.full(N, 0.1)]), p=np.vstack([k, B]),
                 mc=(-1.0, 1.0, 1.0), n_transient=n_transient, n_record=n_record)


def duffing_rkck(nk=512, nB=256, n_transient=1024, n_record=64, events=True):
    k = np.linspace(0.2, 0.3, nk)
    B = np.linspace(0.3, 0.5, nB)
    kk, BB = np.meshgrid(k, B)  # k fastest
    N = nk * nB
    return _base(name="duffing_rkck_%dx%d" % (nk, nB), model=DUFFING, scheme=RKCK45, N=N, h0=1e-2,
                 td=np.vstack([np.zeros(N), np.full(N, 2 * math.pi)]),
                 y0=np.vstack([np.full(N, -0.5), np.full(N, 0.1)]),
                 p=np.vstack([kk.ravel(), BB.ravel()]), mc=(-1.0, 1.0, 1.0), events_on=events,
                 evt_dir=(-1,), evt_tol=(1e-12,), evt_stop=(0,), n_transient=n_transient,
                 n_record=n_record)


def duffing_lyapunov(N=61440, n_transient=1024, n_record=64, c3=1.0):
    """Sec. 7.1.3 (Table 4, the largest of its thread counts): each record
    holds a4 = ln y3 over one period; the exponent is their mean / (2 pi).
    c3 = 0 gives the linear oscillator, whose exponent is -k / 2."""
    k = np.linspace(0.2, 0.3, N)
    B = np.full(N, 0.3)
    return _base(name="duffing_lyapunov_%d" % N, model=DUFFING_LYAPUNOV, scheme=RKCK45, N=N, h0=1e-2,
                 rtol=1e-9, atol=1e-9, td=np.vstack([np.zeros(N), np.full(N, 2 * math.pi)]),
                 y0=np.vstack([np.full(N, -0.5), np.full(N, 0.1), np.ones(N), np.zeros(N)]),
                 p=np.vstack([k, B]), mc=(-1.0, c3, 1.0), n_transient=n_transient, n_record=n_record)


def keller_miksis(npa=512, nf=512, n_transient=1024, n_record=64, pa_max=2.0e5):
    pa = np.linspace(0.0, pa_max, npa)
    f = np.logspace(math.log10(20e3), math.log10(1000e3), nf)
    ff, pp = np.meshgrid(f, pa)  # f fastest
    N = npa * nf
    return _base(name="keller_miksis_%dx%d" % (npa, nf), model=KELLER_MIKSIS, scheme=RKCK45, N=N,
                 h0=1e-2, td=np.vstack([np.zeros(N), np.ones(N)]),
                 y0=np.vstack([np.ones(N), np.zeros(N)]), PA=pp.ravel(), omega=2 * math.pi * ff.ravel(),
                 phys=dict(KM_PHYS), n_transient=n_transient, n_record=n_record)


def keller_miksis_collapse(npa=8, nf=8, n_transient=16, n_record=8, pa_max=2.0e5):
    """The collapse-to-collapse iteration of Sec. 7.2: each slice runs from a
    local maximum of the radius to the next (event y2 = 0 downwards, stop 1,
    tolerance 1e-6), t1 = 1e6 and the Finalization moving t0 to the stop time,
    so a record holds (tau_max, y1_max, tau_min, y1_min) of one collapse.
    Single frequency on the pA x f grid of the benchmark sweep without its
    unforced row (an unforced bubble has no maximum to stop at)."""
    w = keller_miksis(npa + 1, nf, n_transient, n_record, pa_max)
    keep = w["PA"] > 0
    N = int(keep.sum())
    w.update(N=N, PA=w["PA"][keep], omega=w["omega"][keep], y0=np.ascontiguousarray(w["y0"][:, keep]))
    w.update(name="keller_miksis_collapse_%dx%d" % (npa, nf), td=np.vstack([np.zeros(N), np.full(N, 1e6)]),
             events_on=True, evt_dir=(-1,), evt_tol=(1e-6,), evt_stop=(1,), td_mode=TD_T0_TO_T)
    return w


def keller_miksis_dual(nf1=4, nf2=4, n_transient=8, n_record=4):
    """The four-dimensional dual-frequency scan of Sec. 7.2 (Table 5): P_A1 in
    {0.5, 1.1} bar, P_A2 in {0.7, 1.2} bar, f1 and f2 log-spaced in
    [20, 1000] kHz (f2 fastest), theta = 0, iterated collapse to collapse."""
    pa1 = np.array([0.5e5, 1.1e5])
    pa2 = np.array([0.7e5, 1.2e5])
    f = np.logspace(math.log10(20e3), math.log10(1000e3), max(nf1, nf2))
    f1, f2 = f[:nf1], f[:nf2]
    A1, A2, F1, F2 = (x.ravel() for x in np.meshgrid(pa1, pa2, f1, f2, indexing="ij"))
    N = A1.size
    return _base(name="keller_miksis_dual_%d" % N, model=KELLER_MIKSIS, scheme=RKCK45, N=N, h0=1e-2,
                 td=np.vstack([np.zeros(N), np.full(N, 1e6)]), y0=np.vstack([np.ones(N), np.zeros(N)]),
                 PA=A1, omega=2 * math.pi * F1, PA2=A2, omega2=2 * math.pi * F2, phys=dict(KM_PHYS),
                 events_on=True, evt_dir=(-1,), evt_tol=(1e-6,), evt_stop=(1,), td_mode=TD_T0_TO_T,
                 n_transient=n_transient, n_record=n_record)


def valve(N=65536, n_transient=1024, n_record=64, rtol=1e-9):
    q = np.linspace(0.2, 10.0, N)
    v = VALVE_FIXED
    p = np.vstack([np.full(N, v["kappa"]), np.full(N, v["delta"]), np.full(N, v["beta"]), q,
                   np.full(N, v["r"])])
    return _base(name="valve_%d" % N, model=VALVE, scheme=RKCK45, N=N, h0=1e-2, rtol=rtol, atol=rtol,
                 td=np.vstack([np.zeros(N), np.full(N, 1e3)]),
                 y0=np.vstack([np.full(N, 0.2), np.zeros(N), np.full(N, v["delta"])]), p=p,
                 events_on=True, evt_dir=(-1, -1), evt_tol=(1e-6, 1e-6), evt_stop=(1, 0), max_eq=50,
                 td_mode=TD_SHIFT, n_transient=n_transient, n_record=n_record)


def bounce(N=64, n_record=4):
    g = np.linspace(0.5, 2.0, N)
    r = np.linspace(0.5, 0.9, N)
    return _base(name="bounce_%d" % N, model=BOUNCE, scheme=RKCK45, N=N, h0=1e-2, hmax=0.05,
                 td=np.vstack([np.zeros(N), np.full(N, 3.0)]),
                 y0=np.vstack([np.linspace(0.5, 2.0, N), np.zeros(N)]), p=np.vstack([g, r]),
                 events_on=True, evt_dir=(-1,), evt_tol=(1e-12,), evt_stop=(0,), td_mode=TD_T0_TO_T,
                 n_transient=0, n_record=n_record)


def subset(w, idx):
    """The same workload restricted to systems `idx` (sorted, unique)."""
    idx = np.asarray(idx)
    out = dict(w)
    out["N"] = len(idx)
    for key in ("td", "y0", "p"):
        if key in w:
            out[key] = np.ascontiguousarray(w[key][:, idx])
    for key in ("PA", "omega", "PA2", "omega2"):
        if key in w:
            out[key] = np.ascontiguousarray(w[key][idx])
    out["name"] = w["name"] + "_sub%d" % len(idx)
    return out


def sample_indices(N, count, seed=SEED, corners=()):
    """Seeded sample of `count` system indices that includes `corners`."""
    rng = np.random.default_rng(seed)
    base = set(int(c) % N for c in corners)
    rest = rng.choice(N, size=min(N, count + len(base)), replace=False)
    for r in rest:
        if len(base) >= count:
            break
        base.add(int(r))
    return np.array(sorted(base))


def serving_mix(n_requests=2000, rate=1.0, seed=SEED, max_log2_size=16, min_log2_h=4, max_log2_h=10):
    """Poisson stream of sweep requests: (arrival time, model, size, horizon,
    seed of its own parameter stream).  `rate` is requests per second."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    models = rng.choice([DUFFING, KELLER_MIKSIS, VALVE], size=n_requests)
    sizes = np.floor(2.0 ** rng.uniform(0, max_log2_size, size=n_requests)).astype(np.int64)
    horizons = np.floor(2.0 ** rng.uniform(min_log2_h, max_log2_h, size=n_requests)).astype(np.int64)
    seeds = rng.integers(0, 2**31 - 1, size=n_requests)
    return [dict(arrival=float(a), model=int(m), size=max(1, int(s)), horizon=int(h), seed=int(sd))
            for a, m, s, h, sd in zip(arrivals, models, sizes, horizons, seeds)]


def request_inputs(req):
    """Parameters and initial conditions of one serving request, drawn from
    its own seeded stream, uniform in the ranges of the sweep workloads."""
    rng = np.random.default_rng(req["seed"])
    n = req["size"]
    m = req["model"]
    if m == DUFFING:
        w = duffing_rkck(1, 1, 0, 1)
        p = np.vstack([rng.uniform(0.2, 0.3, n), rng.uniform(0.3, 0.5, n)])
        return dict(w, N=n, p=p, td=np.vstack([np.zeros(n), np.full(n, 2 * math.pi)]),
                    y0=np.vstack([np.full(n, -0.5), np.full(n, 0.1)]), n_transient=0,
                    n_record=req["horizon"], events_on=True)
    if m == KELLER_MIKSIS:
        w = keller_miksis(1, 1, 0, 1)
        PA = rng.uniform(0.0, 2.0e5, n)
        f = 10 ** rng.uniform(math.log10(20e3), math.log10(1000e3), n)
        return dict(w, N=n, PA=PA, omega=2 * math.pi * f, td=np.vstack([np.zeros(n), np.ones(n)]),
                    y0=np.vstack([np.ones(n), np.zeros(n)]), n_transient=0, n_record=req["horizon"])
    w = valve(1, 0, 1)
    q = rng.uniform(0.2, 10.0, n)
    v = VALVE_FIXED
    p = np.vstack([np.full(n, v["kappa"]), np.full(n, v["delta"]), np.full(n, v["beta"]), q,
                   np.full(n, v["r"])])
    return dict(w, N=n, p=p, td=np.vstack([np.zeros(n), np.full(n, 1e3)]),
                y0=np.vstack([np.full(n, 0.2), np.zeros(n), np.full(n, v["delta"])]), n_transient=0,
                n_record=req["horizon"])
