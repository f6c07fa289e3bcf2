"""The no-allocation entry point against the solver-object entry point.

ode_run_periods_noalloc serves callers that cannot allocate device memory
(their memory belongs to another allocator's pool, or they cannot afford the
device synchronisation of cudaMalloc / cudaFree): it integrates the caller's
device arrays and keeps the kernel's bookkeeping in a fixed array inside the
library.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as W
from paper_1810_03931_gb300 import odegpu as G

from _runners import DIMS, run_gpu

pytestmark = pytest.mark.gpu


def _settings(w):
    n, P, A, E = DIMS[w["model"]]
    s = G.NoAllocSettings()
    s.model, s.scheme, s.prec = w["model"], w["scheme"], G.ODE_FP64
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
    s.max_steps_per_slice = 10**9
    s.time_limit_s = 300.0
    for i, c in enumerate(w["mc"]):
        s.model_constants[i] = c
    return s


@pytest.mark.parametrize("make", [lambda: W.duffing_rkck(64, 8, 4, 3),
                                  lambda: W.valve(N=256, n_transient=6, n_record=3)])
def test_noalloc_matches_solver_entry_point_on_two_calls(make):
    import torch
    w = make()
    n, P, A, E = DIMS[w["model"]]
    N, n_tr, n_rec = w["N"], w["n_transient"], w["n_record"]
    ref = run_gpu(w, persistent=1)
    cfg = _settings(w)
    stream = torch.cuda.current_stream()
    for call in range(2):
        td = torch.tensor(w["td"], dtype=torch.float64, device="cuda")
        y = torch.tensor(w["y0"], dtype=torch.float64, device="cuda")
        p = torch.tensor(w["p"], dtype=torch.float64, device="cuda")
        acc = torch.zeros((A, N), dtype=torch.float64, device="cuda")
        rec = torch.zeros((n_rec, A + n + 1, N), dtype=torch.float64, device="cuda")
        status = torch.zeros(N, dtype=torch.int32, device="cuda")
        accepted = torch.zeros(N, dtype=torch.int64, device="cuda")
        G.ode_run_periods_noalloc(cfg, N, 0, w["h0"], n_tr, n_rec, td, y, p, acc, rec, status,
                                  accepted, stream)
        torch.cuda.synchronize()
        # the tightest tolerance of the parity tests (1e-12 relative)
        np.testing.assert_allclose(rec.cpu().numpy(), ref["records"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(y.cpu().numpy(), ref["y"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(acc.cpu().numpy(), ref["acc"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(td.cpu().numpy(), ref["td"], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(status.cpu().numpy(), ref["status"])
        # counters restart at zero on every call
        np.testing.assert_array_equal(accepted.cpu().numpy(), ref["nacc"])


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    w = W.duffing_rkck(4, 1, 0, 1)
    cfg = _settings(w)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(G.ODEError) as e:
        G.ode_run_periods_noalloc(cfg, 65537, 0, 1e-2, 0, 1, x, x, x, x)
    assert "65536" in str(e.value)
