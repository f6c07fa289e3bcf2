"""Run one workload (see ``workloads``) through the CUDA library or the oracle.

Both runners take the same seeded inputs.  For Keller-Miksis each side
computes its own coefficients C0..C12 from the physical parameters: the GPU
runner with the library's ``ode_km_coefficients``, the oracle runner with the
oracle's own implementation.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1810_03931_gb300 import odegpu as G
from paper_1810_03931_gb300.sweeps import MODEL_DIMS as DIMS  # n, P, A, E
from paper_1810_03931_gb300.sweeps import km_params as km_params_gpu


def _second(w):
    N = w["N"]
    pa2 = w.get("PA2", np.zeros(N))
    om2 = w.get("omega2", w["omega"])
    return pa2, om2


def km_params_oracle(w):
    ph = w["phys"]
    pa2, om2 = _second(w)
    return O.km_coefficients(w["PA"], w["omega"], PA2=pa2, omega2=om2, theta=0.0, **ph)


def gpu_solver(w, prec=G.ODE_FP64, persistent=0, block=0, device=0):
    n, P, A, E = DIMS[w["model"]]
    s = G.ode_create(w["model"], w["scheme"], prec, w["N"], device)
    G.ode_set_tolerances(s, np.full(n, w["rtol"]), np.full(n, w["atol"]), w["hmax"], w["hmin"],
                         w["grow"], w["shrink"])
    G.ode_set_events(s, int(w["events_on"]), np.array(w["evt_dir"][:E], dtype=np.int32),
                     np.array(w["evt_tol"][:E]), np.array(w["evt_stop"][:E], dtype=np.int32),
                     w["max_eq"])
    if w["mc"]:
        G.ode_set_model_constants(s, np.array(w["mc"], dtype=np.float64))
    G.ode_set_time_domain_mode(s, w["td_mode"])
    G.ode_set_launch(s, block, persistent)
    G.ode_set_time_limit(s, 300.0)
    return s


def gpu_load(s, w, params=None):
    N = w["N"]
    p = params if params is not None else (km_params_gpu(w) if w["model"] == 1 else w["p"])
    n, P, A, E = DIMS[w["model"]]
    G.ode_linear_set(s, 0, 0, N, N, td=np.ascontiguousarray(w["td"], dtype=np.float64),
                     y=np.ascontiguousarray(w["y0"], dtype=np.float64),
                     p=np.ascontiguousarray(p, dtype=np.float64), acc=np.zeros((A, N)),
                     copy_mode=G.ODE_ALL)


def gpu_results(s, w, records=None):
    N = w["N"]
    n, P, A, E = DIMS[w["model"]]
    td, y, p, acc = np.zeros((2, N)), np.zeros((n, N)), np.zeros((P, N)), np.zeros((A, N))
    G.ode_linear_get(s, 0, 0, N, N, td=td, y=y, p=p, acc=acc, copy_mode=G.ODE_ALL)
    status = np.zeros(N, dtype=np.int32)
    nacc = np.zeros(N, dtype=np.int64)
    nrej = np.zeros(N, dtype=np.int64)
    ecnt = np.zeros((E, N), dtype=np.int32)
    G.ode_get_status(s, status, nacc, nrej, ecnt)
    out = dict(td=td, y=y, acc=acc, status=status, nacc=nacc, nrej=nrej, ecnt=ecnt)
    if records is not None:
        out["records"] = records
    return out


def run_gpu(w, prec=G.ODE_FP64, persistent=0, block=0, record=True, n_transient=None, n_record=None,
            autotune=False):
    """autotune: pick the launch shape with the library's autotuner on a short
    trial first, as the benchmark does (the trial leaves the state as loaded)."""
    n_tr = w["n_transient"] if n_transient is None else n_transient
    n_rec = w["n_record"] if n_record is None else n_record
    n, P, A, E = DIMS[w["model"]]
    s = gpu_solver(w, prec, persistent, block)
    try:
        gpu_load(s, w)
        if autotune:
            G.ode_autotune(s, w["h0"], 4)
        rec = np.zeros((n_rec, A + n + 1, w["N"])) if record and n_rec > 0 else None
        G.ode_run_periods(s, w["h0"], n_tr, n_rec, rec)
        G.ode_synchronize(s)
        return gpu_results(s, w, rec)
    finally:
        G.ode_destroy(s)


def run_oracle(w, nthreads=8, record=True, n_transient=None, n_record=None, **cfg_over):
    return O.run_workload(w, nthreads, record, n_transient, n_record, **cfg_over)
