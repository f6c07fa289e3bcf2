"""The no-allocation entry point against the solver-object entry point.

ode_run_periods_noalloc serves callers that cannot allocate device memory
(their memory belongs to another allocator's pool, or they cannot afford the
device synchronisation of cudaMalloc / cudaFree): it integrates the caller's
device arrays and keeps the kernel's bookkeeping in a fixed array inside the
library.  Sizes that are odd or not a multiple of the 128-thread block stress
the layout of that array (each section must stay aligned for its type); both
schemes and both precisions go through it.  This file is collected last so
that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as W
from paper_1810_03931_gb300 import odegpu as G
from paper_1810_03931_gb300.sweeps import settings_for

from _runners import DIMS, run_gpu
from test_parity_gpu import _compare_records, _nonchaotic

pytestmark = pytest.mark.gpu

CASES = {
    "duffing_rkck45_512": (lambda: W.duffing_rkck(64, 8, 4, 3), G.ODE_FP64),
    "valve_rkck45_256": (lambda: W.valve(N=256, n_transient=6, n_record=3), G.ODE_FP64),
    "duffing_rkck45_odd33": (lambda: W.duffing_rkck(33, 1, 3, 2), G.ODE_FP64),
    "duffing_rkck45_odd1025": (lambda: W.duffing_rkck(41, 25, 3, 2), G.ODE_FP64),
    "duffing_rk4_1000": (lambda: W.duffing_rk4(N=1000, n_transient=2, n_record=2), G.ODE_FP64),
    "valve_fp32rhs_odd63": (lambda: W.valve(N=63, n_transient=4, n_record=2), G.ODE_FP32_RHS),
}


def _noalloc_run(w, prec):
    import torch
    n, P, A, E = DIMS[w["model"]]
    N, n_tr, n_rec = w["N"], w["n_transient"], w["n_record"]
    cfg = settings_for(w, prec)
    td = torch.tensor(w["td"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y0"], dtype=torch.float64, device="cuda")
    p = torch.tensor(w["p"], dtype=torch.float64, device="cuda")
    acc = torch.zeros((A, N), dtype=torch.float64, device="cuda")
    rec = torch.zeros((n_rec, A + n + 1, N), dtype=torch.float64, device="cuda")
    status = torch.zeros(N, dtype=torch.int32, device="cuda")
    accepted = torch.zeros(N, dtype=torch.int64, device="cuda")
    G.ode_run_periods_noalloc(cfg, N, 0, w["h0"], n_tr, n_rec, td, y, p, acc, rec, status, accepted,
                              torch.cuda.current_stream())
    torch.cuda.synchronize()
    return dict(records=rec.cpu().numpy(), y=y.cpu().numpy(), acc=acc.cpu().numpy(),
                td=td.cpu().numpy(), status=status.cpu().numpy(), nacc=accepted.cpu().numpy())


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_solver_entry_point_on_two_calls(case):
    make, prec = CASES[case]
    w = make()
    ref = run_gpu(w, prec=prec, persistent=1)
    for call in range(2):
        out = _noalloc_run(w, prec)
        # the tightest tolerance of the parity tests (1e-12 relative)
        for key in ("records", "y", "acc", "td"):
            np.testing.assert_allclose(out[key], ref[key], rtol=1e-12, atol=1e-12, err_msg=key)
        np.testing.assert_array_equal(out["status"], ref["status"])
        # counters restart at zero on every call
        np.testing.assert_array_equal(out["nacc"], ref["nacc"])


def test_noalloc_odd_size_matches_the_oracle():
    """33 systems (odd, a partial block): against the CPU oracle at the
    acceptance of the RKCK45 parity tests (event maxima and end states within
    1e-8 on well-conditioned points, counts exact)."""
    w = W.duffing_rkck(33, 1, 3, 2)
    mask, o = _nonchaotic(w, w["n_transient"], w["n_record"], cont_rows=(4, 5, 7, 8), rtol=1e-10)
    assert mask.sum() >= 30
    g = _noalloc_run(w, G.ODE_FP64)
    assert np.all(g["status"] == 1)
    _compare_records(g, o, mask, 7, 2, tol=1e-8, exact_rows=(6, 9))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    w = W.duffing_rkck(4, 1, 0, 1)
    cfg = settings_for(w)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(G.ODEError) as e:
        G.ode_run_periods_noalloc(cfg, 65537, 0, 1e-2, 0, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                  x.data_ptr())
    assert "65536" in str(e.value)
    # short tensors are refused by the binding before the library is called
    with pytest.raises(G.ODEError) as e:
        G.ode_run_periods_noalloc(cfg, 4, 0, 1e-2, 0, 1, x, x, x, x)
    assert "elements" in str(e.value)
