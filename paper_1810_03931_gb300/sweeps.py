"""Marshalling of a seeded sweep description (``workloads``) into the
library's calls: model dimensions, Keller-Miksis coefficients through the
library's ``ode_km_coefficients`` (Eqs. 16-28), and the settings block of the
allocation-free call and the serving loop.  No arithmetic of the method runs
here; the coefficients come from the C ABI.
"""
from __future__ import annotations

import numpy as np

from . import odegpu as G

# (n, P, A, E) per model id: state dimension, parameters, accessories, events
MODEL_DIMS = G.MODEL_DIMS


def km_params(w):
    """Coefficients C0..C12 [13][N] of a Keller-Miksis sweep from its physical
    parameters (pressure amplitudes, angular frequencies), one library call
    per system."""
    ph = w["phys"]
    N = w["N"]
    pa2 = w.get("PA2", np.zeros(N))
    om2 = w.get("omega2", w["omega"])
    P = np.zeros((13, N))
    for i in range(N):
        P[:, i] = G.ode_km_coefficients(w["PA"][i], pa2[i], w["omega"][i], om2[i], 0.0, ph["RE"],
                                        ph["Pinf"], ph["pV"], ph["sigma"], ph["mu"], ph["rho"], ph["cL"],
                                        ph["gamma"])
    return P


def params(w):
    """The parameter array [P][N] the library takes for sweep w."""
    return km_params(w) if w["model"] == G.ODE_KELLER_MIKSIS else w["p"]


def settings_for(w, prec=G.ODE_FP64, max_steps_per_slice=10**9, time_limit_s=300.0):
    """The ``ode_noalloc_settings`` block of sweep w (solver settings of
    Secs. 6.5-6.6 and the time-domain mode)."""
    n, P, A, E = MODEL_DIMS[w["model"]]
    s = G.NoAllocSettings()
    s.model, s.scheme, s.prec = w["model"], w["scheme"], prec
    for i in range(4):
        s.rtol[i] = w["rtol"]
        s.atol[i] = w["atol"]
    s.h_max, s.h_min, s.grow_limit, s.shrink_limit = w["hmax"], w["hmin"], w["grow"], w["shrink"]
    s.events_enabled = int(w["events_on"])
    for j in range(min(E, 2)):
        s.direction[j] = w["evt_dir"][j]
        s.tolerance[j] = w["evt_tol"][j]
        s.stop_count[j] = w["evt_stop"][j]
    s.max_steps_in_zone = w["max_eq"]
    s.time_domain_mode = w["td_mode"]
    s.max_steps_per_slice = max_steps_per_slice
    s.time_limit_s = time_limit_s
    for i, c in enumerate(w["mc"]):
        s.model_constants[i] = c
    return s
