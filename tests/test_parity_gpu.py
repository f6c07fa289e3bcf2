"""GPU (CUDA library, through the C ABI) against the CPU oracle, element by
element on the same seeded inputs.

Acceptance:
  * RK4 binary64 final states and records: 1e-12 relative (atol 1e-12).
  * RKCK45 accessories, event points and Poincare points: 100 x rtol on
    well-conditioned (non-chaotic) parameter points.  A point qualifies when
    the oracle at rtol and at rtol / 10 agrees on its recorded continuous
    quantities (end state and event-located maxima) within the acceptance
    tolerance itself (Duffing: 10 x rtol suffices; Keller-Miksis collapses
    amplify local errors so that its global error is already ~10-100 x rtol).
  * Where an event ends a slice or changes the state (valve impacts), the
    located point is only fixed to the event tolerance, so the acceptance is
    max(100 x rtol, 10 x event tolerance).
  * Discrete accessories (max / min over accepted points) may pick the other
    of two near-equal samples; their times are then checked for validity
    (the value agrees) instead of equality.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from paper_1810_03931_gb300 import odegpu as G

from _runners import DIMS, gpu_load, gpu_results, gpu_solver, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def _report(line):
    """Print a parity figure (mask fractions, statistics) and, when
    ODEGPU_PARITY_REPORT names a file, append it there."""
    print(line)
    path = os.environ.get("ODEGPU_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


def _rel_close(a, b, rtol, atol):
    return np.abs(a - b) <= atol + rtol * np.abs(b)


def _nonchaotic(w, n_tr, n_rec, cont_rows, rtol, agree=None):
    """Mask of systems whose continuous records agree at rtol and rtol/10
    within `agree` (default 10 x rtol)."""
    agree = 10 * rtol if agree is None else agree
    r1 = run_oracle(w, NTHREADS, n_transient=n_tr, n_record=n_rec)
    r2 = run_oracle(w, NTHREADS, n_transient=n_tr, n_record=n_rec, rtol=rtol / 10, atol=rtol / 10)
    ok = np.ones(w["N"], dtype=bool)
    for row in cont_rows:
        ok &= np.all(_rel_close(r1["records"][:, row], r2["records"][:, row], agree, agree), axis=0)
    return ok, r1


def _compare_records(g, o, mask, A, n, tol, discrete_pairs=((0, 1), (2, 3)), exact_rows=()):
    """Compare records of `mask` systems; returns the number compared."""
    rg, ro = g["records"][:, :, mask], o["records"][:, :, mask]
    R = A + n + 1
    for row in range(R):
        if row in exact_rows:
            np.testing.assert_array_equal(rg[:, row], ro[:, row], err_msg="row %d" % row)
            continue
        times = {t for _, t in discrete_pairs}
        if row in times:
            continue
        np.testing.assert_array_less(np.abs(rg[:, row] - ro[:, row]), tol * (1 + np.abs(ro[:, row])),
                                     err_msg="record row %d" % row)
    for vrow, trow in discrete_pairs:
        same_t = np.abs(rg[:, trow] - ro[:, trow]) <= tol * (1 + np.abs(ro[:, trow]))
        same_v = np.abs(rg[:, vrow] - ro[:, vrow]) <= tol * (1 + np.abs(ro[:, vrow]))
        # a different time is valid only when the sampled values tie
        assert np.all(same_t | same_v)
    return int(mask.sum())


# ---------------------------------------------------------------------------
# Duffing RK4 (the Poincare loop of Sec. 7.1.1 with accessories), full size.
# ---------------------------------------------------------------------------
def test_duffing_rk4_full_size_parity():
    w = W.duffing_rk4()
    g = run_gpu(w)
    o = run_oracle(w, NTHREADS)
    assert np.all(g["status"] == W.RK4 + 1) and np.all(o["status"] == 1)
    np.testing.assert_array_equal(g["nacc"], o["nacc"])
    np.testing.assert_array_equal(g["nacc"], 96 * 1000)
    assert np.all(_rel_close(g["y"], o["y"], 1e-12, 1e-12))
    rg, ro = g["records"], o["records"]
    for row in (0, 2, 4, 7, 8):  # max, min, event-acc init value, Poincare point
        assert np.all(_rel_close(rg[:, row], ro[:, row], 1e-12, 1e-12)), row
    np.testing.assert_array_equal(rg[:, 9], ro[:, 9])  # end time: t1 exactly
    for vrow, trow in ((0, 1), (2, 3)):
        same_t = rg[:, trow] == ro[:, trow]
        assert np.all(same_t | _rel_close(rg[:, vrow], ro[:, vrow], 1e-12, 1e-12))


def test_duffing_rk4_mixed_time_domains_parity():
    """The block-shared forcing table serves the systems whose slice matches
    the grid it was built for; the others rotate their own forcing anchor.
    Every fourth system here has another time domain (and so another step
    size and grid); the block's first system alternates between the two
    kinds, so both paths run in the same warps.  Both kinds match the oracle
    at the RK4 acceptance (1e-12 relative)."""
    w = W.duffing_rk4(N=320, n_transient=3, n_record=2)
    td = w["td"].copy()
    td[1, 1::4] = 1.5 * math.pi   # shorter slices, other steps
    td[0, 64::128] = 0.25         # some blocks' first system off the common grid
    w = dict(w, td=td)
    o = run_oracle(w, NTHREADS)
    for persistent in (0, 1):
        g = run_gpu(w, persistent=persistent, block=64)
        np.testing.assert_array_equal(g["nacc"], o["nacc"])
        assert np.all(_rel_close(g["y"], o["y"], 1e-12, 1e-12))
        for row in (0, 2, 7, 8):
            assert np.all(_rel_close(g["records"][:, row], o["records"][:, row], 1e-12, 1e-12)), row


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_duffing_rk4_launch_forms_identical(persistent):
    w = W.duffing_rk4(N=333, n_transient=2, n_record=2)
    base = run_gpu(w, persistent=0, block=64)
    other = run_gpu(w, persistent=persistent, block=128)
    for key in ("y", "acc", "records", "nacc"):
        np.testing.assert_array_equal(base[key], other[key])


# ---------------------------------------------------------------------------
# Duffing RKCK45 with the local-maximum event (Sec. 7.1.2), cfg of the bench.
# ---------------------------------------------------------------------------
def _duffing_rkck_small(nk=32, nB=16, n_tr=20, n_rec=8):
    w = W.duffing_rkck(nk, nB, n_tr, n_rec)
    return w


def test_duffing_rkck_event_parity_grid():
    w = _duffing_rkck_small()
    A, n = 7, 2
    mask, o = _nonchaotic(w, w["n_transient"], w["n_record"], cont_rows=(4, 5, 7, 8), rtol=1e-10)
    assert mask.mean() > 0.5
    g = run_gpu(w)
    assert np.all(g["status"] == 1)
    # event counts are integers: compared exactly on non-chaotic points
    cnt = _compare_records(g, o, mask, A, n, tol=1e-8, exact_rows=(6, 9))
    assert cnt > 0
    # step counts agree closely (the step-size sequences are the same up to
    # rounding of the error estimate)
    ratio = g["nacc"][mask] / o["nacc"][mask]
    assert np.all(np.abs(ratio - 1) < 1e-3)


def test_duffing_rkck_full_size_sampled():
    """The bench workload at full size (2^17 systems, 1024 + 64 periods), in the
    launch form the bench's autotuner picks; sampled systems replayed one by one
    by the oracle."""
    w = W.duffing_rkck()
    g = run_gpu(w, autotune=True)
    assert np.all(np.isin(g["status"], [1]))
    idx = W.sample_indices(w["N"], 256, corners=(0, 511, w["N"] - 512, w["N"] - 1))
    ws = W.subset(w, idx)
    mask, o = _nonchaotic(ws, w["n_transient"], w["n_record"], cont_rows=(4, 5, 7, 8), rtol=1e-10)
    gs = {k: (v[..., idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    _report("duffing_rkck full size: well-conditioned mask keeps %d of %d sampled systems"
            % (mask.sum(), len(idx)))
    assert mask.sum() >= 230
    _compare_records(gs, o, mask, 7, 2, tol=1e-8, exact_rows=(6, 9))
    # every system integrated every period
    assert np.all(g["nacc"] > 1088 * 50)


# ---------------------------------------------------------------------------
# Duffing with its polar linearisation (Sec. 7.1.3): per-period ln y3 with the
# radius reset by the Finalization hook.
# ---------------------------------------------------------------------------
def test_duffing_lyapunov_parity():
    w = W.duffing_lyapunov(N=320, n_transient=12, n_record=6)
    A, n = 5, 4
    # continuous records: ln-stretch a4 and the end state (y3 is 1 after reset)
    # agreement at 100 x rtol: ln y3 integrates the error over a whole period
    mask, o = _nonchaotic(w, w["n_transient"], w["n_record"], cont_rows=(4, 5, 6, 8), rtol=1e-9,
                          agree=1e-7)
    assert mask.mean() > 0.5
    g = run_gpu(w)
    assert np.all(g["status"] == 1)
    np.testing.assert_array_equal(g["records"][:, A + 2], 1.0)
    _compare_records(g, o, mask, A, n, tol=1e-7, exact_rows=(9,))
    ratio = g["nacc"][mask] / o["nacc"][mask]
    assert np.all(np.abs(ratio - 1) < 1e-3)


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_duffing_lyapunov_launch_forms_identical(persistent):
    w = W.duffing_lyapunov(N=200, n_transient=3, n_record=2)
    base = run_gpu(w, persistent=0, block=64)
    other = run_gpu(w, persistent=persistent, block=96)
    for key in ("y", "acc", "records", "nacc"):
        np.testing.assert_array_equal(base[key], other[key])


def test_duffing_lyapunov_linear_oscillator_exponent():
    # c3 = 0: the exponent of x'' + k x' + x = B cos t is -k / 2; over n
    # periods the per-time mean of ln y3 carries a bounded term / (n T)
    w = W.duffing_lyapunov(N=64, n_transient=0, n_record=200, c3=0.0)
    g = run_gpu(w)
    k = w["p"][0]
    lam = g["records"][:, 4].sum(axis=0) / (200 * 2 * math.pi)
    np.testing.assert_allclose(lam, -k / 2, rtol=0, atol=5e-4)


def test_duffing_lyapunov_full_size_sampled():
    """The Lyapunov sweep at full size (61440 systems, 1024 + 64 periods) in
    the persistent launch; sampled systems replayed by the oracle.  The
    tangent angle of an orbit with complex Floquet multipliers is neutrally
    stable, so its error (and that of the per-period ln-stretch, which
    depends on it) grows with the horizon: after 1088 periods the oracle at
    rtol and at rtol / 10 differs there by ~1e-6.  Those two rows are held to
    10 x that spread; the oscillator's own state and extrema to 100 x rtol."""
    w = W.duffing_lyapunov()
    g = run_gpu(w, autotune=True)
    assert np.all(g["status"] == 1)
    idx = W.sample_indices(w["N"], 256, corners=(0, 1, w["N"] - 2, w["N"] - 1))
    ws = W.subset(w, idx)
    mask, o = _nonchaotic(ws, w["n_transient"], w["n_record"], cont_rows=(5, 6), rtol=1e-9, agree=1e-7)
    o2 = run_oracle(ws, NTHREADS, rtol=1e-10, atol=1e-10)
    _report("duffing_lyapunov full size: well-conditioned mask keeps %d of %d sampled systems"
            % (mask.sum(), len(idx)))
    assert mask.sum() >= 192
    rg, ro, ro2 = g["records"][:, :, idx][:, :, mask], o["records"][:, :, mask], o2["records"][:, :, mask]
    for row in (0, 2, 5, 6):  # max, min of y1; y1, y2
        np.testing.assert_array_less(np.abs(rg[:, row] - ro[:, row]), 1e-7 * (1 + np.abs(ro[:, row])))
    np.testing.assert_array_equal(rg[:, 7], 1.0)
    np.testing.assert_array_equal(rg[:, 9], ro[:, 9])
    # ln-stretch; reduced angle (differences taken modulo 2 pi)
    dang = lambda a, b: np.abs(np.remainder(a - b + math.pi, 2 * math.pi) - math.pi)
    for row, diff in ((4, lambda a, b: np.abs(a - b)), (8, dang)):
        spread = np.max(diff(ro2[:, row], ro[:, row]))
        assert spread < 1e-4
        np.testing.assert_array_less(diff(rg[:, row], ro[:, row]), max(10 * spread, 1e-7))
    # the exponents of the whole sweep are finite and, on the sampled
    # periodic points, negative
    lam = g["records"][:, 4].mean(axis=0) / (2 * math.pi)
    assert np.all(np.isfinite(lam))
    assert np.all(lam[idx][mask] < 0)


# ---------------------------------------------------------------------------
# Keller-Miksis (Sec. 2.2, single frequency), grid corners and interior.
# ---------------------------------------------------------------------------
def test_keller_miksis_parity():
    w = W.keller_miksis(6, 6, 4, 4)
    A, n = 4, 2
    mask, o = _nonchaotic(w, 4, 4, cont_rows=(4, 5), rtol=1e-10, agree=1e-8)
    g = run_gpu(w)
    assert np.all(g["status"] == 1)
    assert mask.sum() >= 24
    _compare_records(g, o, mask, A, n, tol=1e-8, exact_rows=(6,))
    # the unforced column (pA = 0) stays at the equilibrium radius
    pa0 = w["PA"] == 0
    assert np.all(np.abs(g["records"][:, 4, pa0] - 1.0) < 1e-8)


@pytest.mark.parametrize("make", [lambda: W.keller_miksis_collapse(6, 6, 6, 4),
                                  lambda: W.keller_miksis_dual(3, 3, 4, 3)],
                         ids=["collapse_iteration", "dual_frequency"])
def test_keller_miksis_collapse_protocols(make):
    """Collapse-to-collapse iteration (event stop at each maximum, t0 moved to
    the stop time, t1 = 1e6), single and dual frequency (Sec. 7.2).  The
    located maxima are fixed to the event tolerance 1e-6, so the acceptance is
    100 x that tolerance on well-conditioned points."""
    w = make()
    tol = 100 * w["evt_tol"][0]
    mask, o = _nonchaotic(w, w["n_transient"], w["n_record"], cont_rows=(4, 5, 6), rtol=1e-10, agree=tol)
    g = run_gpu(w)
    assert np.all(g["status"] == G.ODE_ST_EVENT_STOP)
    assert mask.sum() >= w["N"] // 3
    # each record is one collapse: it starts at a maximum, so y2 ~ 0 at both ends
    assert np.all(np.abs(g["records"][:, 5]) <= w["evt_tol"][0])
    _compare_records(g, o, mask, 4, 2, tol=tol)


@pytest.mark.parametrize("make", [
    lambda: W.keller_miksis_collapse(255, 256, n_transient=16, n_record=8),
    lambda: W.keller_miksis_dual(128, 128, n_transient=16, n_record=8)],
    ids=["collapse_iteration_65280", "dual_frequency_table5_65536"])
def test_keller_miksis_protocols_bench_size_sampled(make):
    """The collapse and dual-frequency protocols at the benchmark's sizes in the
    autotuned launch shape; sampled systems (grid corners included) replayed one by one
    by the oracle and compared on well-conditioned points at 100 x the event
    tolerance."""
    w = make()
    g = run_gpu(w, autotune=True)
    assert np.all(g["status"] == G.ODE_ST_EVENT_STOP)
    idx = W.sample_indices(w["N"], 256, corners=(0, 255, w["N"] - 256, w["N"] - 1))
    ws = W.subset(w, idx)
    tol = 100 * w["evt_tol"][0]
    mask, o = _nonchaotic(ws, w["n_transient"], w["n_record"], cont_rows=(4, 5, 6), rtol=1e-10, agree=tol)
    gs = {k: (v[..., idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    _report("%s: well-conditioned mask keeps %d of %d sampled systems" % (w["name"], mask.sum(), len(idx)))
    assert mask.sum() >= 192
    _compare_records(gs, o, mask, 4, 2, tol=tol)


# ---------------------------------------------------------------------------
# Pressure relief valve with two events, impact action and equilibrium stop
# (Sec. 7.3), per-sweep and persistent launches.
# ---------------------------------------------------------------------------
def _valve_stable(w, o, o2, tol):
    """Systems whose stop reasons, impact counts, end states and iteration
    durations agree between two oracle runs (e.g. at rtol and at rtol / 10)."""
    stable = np.all(o["records"][:, 4] == o2["records"][:, 4], axis=0) & (o["status"] == o2["status"])
    stable &= np.all(_rel_close(o["records"][:, 5:8], o2["records"][:, 5:8], tol, tol), axis=(0, 1))
    d1, d2 = np.diff(o["records"][:, 8], axis=0), np.diff(o2["records"][:, 8], axis=0)
    stable &= np.all(_rel_close(d1, d2, tol, tol), axis=0)
    return stable


def _valve_well_conditioned(w, tol):
    """Valve systems whose stop reasons, impact counts and end states are
    insensitive both to the integration tolerance (oracle at rtol and at
    rtol / 10) and to the event tolerance (oracle at tol_E and tol_E / 100):
    an event that ends a slice or changes the state is located only to
    |F| <= tol_E, and near grazing impacts that freedom alone can shift which
    iteration an impact falls in.  Returns the mask and the oracle run."""
    o = run_oracle(w, NTHREADS)
    o2 = run_oracle(w, NTHREADS, rtol=w["rtol"] / 10, atol=w["atol"] / 10)
    o3 = run_oracle(w, NTHREADS, evt_tol=tuple(x / 100 for x in w["evt_tol"]))
    return _valve_stable(w, o, o2, tol) & _valve_stable(w, o, o3, tol), o


def _valve_records_match(rg, ro, tol):
    """Records [iteration, row] of one system agree: impact counts exactly;
    maximum, Poincare point and the duration of each iteration within tol
    (relative + absolute).  The valve is autonomous, so the position along a
    periodic orbit is neutrally stable and the absolute time of the n-th
    maximum drifts with every local error (linearly, never damped); the
    durations of the iterations are what the dynamics fix."""
    if not np.array_equal(rg[:, 4], ro[:, 4]):
        return False
    rows = [0, 5, 6, 7]
    if not np.all(np.abs(rg[:, rows] - ro[:, rows]) <= tol * (1 + np.abs(ro[:, rows]))):
        return False
    dg, do = np.diff(rg[:, 8]), np.diff(ro[:, 8])
    return bool(np.all(np.abs(dg - do) <= tol * (1 + np.abs(do))))


def _valve_compare(g, o, stable, tol, max_shift=4):
    """GPU against oracle on well-conditioned valve systems.  A system on a
    periodic orbit (period p iterations) may leave the 1024-iteration
    transient in another phase than the oracle does -- which of the p
    iterations comes first is set by the whole transient, and the oracle's
    own reruns at rtol / 10 and tol_E / 100 can agree on it by chance.  Such
    a system is accepted when its records equal the oracle's shifted by
    s <= max_shift iterations (the same orbit, entered one phase apart);
    the number of them is reported."""
    np.testing.assert_array_equal(g["status"][stable], o["status"][stable])
    shifted = 0
    for i in np.where(stable)[0]:
        rg, ro = g["records"][:, :, i], o["records"][:, :, i]
        if _valve_records_match(rg, ro, tol):
            continue
        ok = any(_valve_records_match(rg[sft:], ro[:-sft], tol) or _valve_records_match(rg[:-sft], ro[sft:], tol)
                 for sft in range(1, max_shift + 1))
        if not ok:
            rows = [0, 5, 6, 7]
            diff = np.abs(rg[:, rows] - ro[:, rows]) / (1 + np.abs(ro[:, rows]))
            dd = np.abs(np.diff(rg[:, 8]) - np.diff(ro[:, 8])) / (1 + np.abs(np.diff(ro[:, 8])))
            raise AssertionError("system %d: records differ from the oracle beyond a phase shift: impacts equal "
                                 "%s, max rel diff of rows 0,5,6,7 %s, of durations %.3e" % (
                                     i, np.array_equal(rg[:, 4], ro[:, 4]), diff.max(axis=0), dd.max()))
        shifted += 1
    dev = np.max(np.abs(g["records"][:, 5:8, stable] - o["records"][:, 5:8, stable]))
    print("valve: %d points compared, %d on the oracle's periodic orbit one or more iterations out of "
          "phase; max |end state - oracle| = %.3e" % (stable.sum(), shifted, dev))
    return shifted


@pytest.mark.parametrize("persistent", [0, 1])
def test_valve_parity(persistent):
    """Two events (maximum with stop 1, impact with action), located to 1e-10
    so that the location error is below the 100 x rtol acceptance."""
    w = W.valve(N=96, n_transient=30, n_record=10)
    w = dict(w, evt_tol=(1e-10, 1e-10))
    o = run_oracle(w, NTHREADS)
    o2 = run_oracle(w, NTHREADS, rtol=1e-10, atol=1e-10)
    tol = 100 * w["rtol"]
    stable = _valve_stable(w, o, o2, tol)
    assert stable.sum() >= 80
    g = run_gpu(w, persistent=persistent)
    _valve_compare(g, o, stable, tol)


@pytest.mark.parametrize("rtol", [1e-9, 1e-10], ids=["rtol1e-9", "paper_rtol1e-10"])
def test_valve_parity_paper_event_tolerance(rtol):
    """The paper's event tolerance 1e-6 (Sec. 6.6): a located point is fixed
    only to |F| <= 1e-6, so the acceptance is 100 x that tolerance; at the
    benchmark's rtol 1e-9 and at the paper's own valve run, rtol = atol =
    1e-10 (Sec. 7.3)."""
    w = W.valve(N=96, n_transient=30, n_record=10, rtol=rtol)
    o = run_oracle(w, NTHREADS)
    o2 = run_oracle(w, NTHREADS, rtol=rtol / 10, atol=rtol / 10)
    tol = 100 * w["evt_tol"][0]
    stable = _valve_stable(w, o, o2, tol)
    assert stable.sum() >= 75
    g = run_gpu(w, persistent=1)
    _valve_compare(g, o, stable, tol)


def test_cluster_order_keeps_results_per_system():
    """Reordering the systems (here: shuffled, then put in the library's
    clustering order) changes which lanes share a warp but no system's
    result."""
    w = W.valve(N=256, n_transient=4, n_record=2)
    ws = W.subset(w, np.random.default_rng(3).permutation(w["N"]))
    perm = G.ode_cluster_order(ws["p"][3:4])  # the swept flow rate q
    wc = W.subset(ws, perm)
    for persistent in (0, 1, 2):
        gs = run_gpu(ws, persistent=persistent)
        gc = run_gpu(wc, persistent=persistent)
        for key in ("y", "acc", "nacc", "status"):
            np.testing.assert_array_equal(gc[key], gs[key][..., perm], err_msg=key)
        np.testing.assert_array_equal(gc["records"], gs["records"][..., perm])


def test_valve_equilibrium_stop_high_flow_rate():
    """q > 8.5 settles to the equilibrium inside the event-0 zone and stops
    after MaximumIterationForEquilibrium = 50 steps (Sec. 4, Sec. 7.3)."""
    w = W.valve(N=16, n_transient=240, n_record=10)
    p = w["p"].copy()
    p[3] = np.linspace(9.0, 10.0, 16)
    w = dict(w, p=p)
    g = run_gpu(w, persistent=1)
    o = run_oracle(w, NTHREADS)
    assert np.all(o["status"] == G.ODE_ST_EQUILIBRIUM)
    np.testing.assert_array_equal(g["status"], o["status"])
    # each recorded iteration ends 50 steps after entering the zone
    np.testing.assert_allclose(g["records"][:, 5:8], o["records"][:, 5:8], rtol=1e-7, atol=1e-7)
    q, d = p[3], w["p"][1][0]
    y1 = g["y"][0]
    np.testing.assert_allclose(y1 * np.sqrt(y1 + d), q, rtol=1e-4)


def test_valve_full_size_sampled():
    """The valve sweep at full size (2^16 systems, 1024 + 64 iterations, both
    events, impacts, equilibrium stops) in the autotuned launch form; sampled
    systems (corners included) replayed by the oracle one by one."""
    w = W.valve()
    s = gpu_solver(w)
    try:
        gpu_load(s, w)
        bs, pers, _ = G.ode_autotune(s, w["h0"], 2)
        n_rec = w["n_record"]
        rec = np.zeros((n_rec, 9, w["N"]))
        G.ode_run_periods(s, w["h0"], w["n_transient"], n_rec, rec)
        G.ode_synchronize(s)
        g = gpu_results(s, w, rec)
    finally:
        G.ode_destroy(s)
    idx = W.sample_indices(w["N"], 256, corners=(0, w["N"] // 2, w["N"] - 1))
    ws = W.subset(w, idx)
    gs = {k: (v[..., idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    tol = 100 * w["evt_tol"][0]
    stable, o = _valve_well_conditioned(ws, tol)
    assert stable.sum() >= 160
    shifted = _valve_compare(gs, o, stable, tol)
    _report("valve full size: well-conditioned mask keeps %d of %d sampled systems; %d of them on the "
            "oracle's periodic orbit in another phase" % (stable.sum(), len(idx), shifted))
    assert shifted <= stable.sum() // 20
    # the high-flow-rate end of the sweep rests at the equilibrium (Sec. 7.3)
    assert np.all(g["status"][w["p"][3] > 9.0] == G.ODE_ST_EQUILIBRIUM)


def test_keller_miksis_bench_size_sampled():
    """The Keller-Miksis sweep of the bench (2^18 systems, 16 + 16 acoustic
    periods) in the autotuned launch form; sampled systems replayed by the
    oracle (C0..C12 computed independently on each side)."""
    w = W.keller_miksis(n_transient=16, n_record=16)
    s = gpu_solver(w)
    try:
        gpu_load(s, w)
        G.ode_autotune(s, w["h0"], 1)
        rec = np.zeros((16, 7, w["N"]))
        G.ode_run_periods(s, w["h0"], 16, 16, rec)
        G.ode_synchronize(s)
        g = gpu_results(s, w, rec)
    finally:
        G.ode_destroy(s)
    assert np.all(g["status"] == 1)
    idx = W.sample_indices(w["N"], 256, corners=(0, 511, w["N"] - 512, w["N"] - 1))
    ws = W.subset(w, idx)
    mask, o = _nonchaotic(ws, 16, 16, cont_rows=(4, 5), rtol=1e-10, agree=1e-8)
    gs = {k: (v[..., idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    _report("keller_miksis full size: well-conditioned mask keeps %d of %d sampled systems"
            % (mask.sum(), len(idx)))
    assert mask.sum() >= 160
    _compare_records(gs, o, mask, 4, 2, tol=1e-8, exact_rows=(6,))


# ---------------------------------------------------------------------------
# Bouncing ball: impact law against its closed form on the GPU too.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", [W.RK4, W.RKCK45])
def test_bounce_closed_form_on_gpu(scheme):
    N = 8
    g0, r0, h0 = 1.0, 0.8, 1.0
    w = W._base(name="ball", model=W.BOUNCE, scheme=scheme, N=N, h0=0.01, hmax=0.05,
                td=np.vstack([np.zeros(N), np.full(N, 12.0)]), y0=np.vstack([np.full(N, h0), np.zeros(N)]),
                p=np.vstack([np.full(N, g0), np.full(N, r0)]), events_on=True, evt_dir=(-1,),
                evt_tol=(1e-12,), evt_stop=(0,), n_transient=0, n_record=1)
    g = run_gpu(w)
    t, v, times = math.sqrt(2 * h0 / g0), math.sqrt(2 * g0 * h0), []
    while t < 12.0:
        times.append((t, -v))
        t += 2 * r0 * v / g0
        v *= r0
    np.testing.assert_array_equal(g["ecnt"][0], len(times))
    np.testing.assert_allclose(g["acc"][4], times[-1][0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(g["acc"][5], times[-1][1], rtol=1e-9)


# ---------------------------------------------------------------------------
# Binary32 right-hand side: the error against the binary64 oracle is measured
# and reported (no tolerance is claimed); the run must complete.
# ---------------------------------------------------------------------------
def test_fp32_rhs_duffing_and_valve_report(tmp_path):
    rows = []
    for w in (W.duffing_rkck(16, 8, 10, 4), W.valve(N=64, n_transient=10, n_record=4)):
        o = run_oracle(w, NTHREADS)
        g = run_gpu(w, prec=G.ODE_FP32_RHS)
        A, n = DIMS[w["model"]][2], DIMS[w["model"]][0]
        assert np.all(np.isfinite(g["records"]))
        assert np.all(g["status"] > 0)
        err = np.max(np.abs(g["records"][:, A:A + n] - o["records"][:, A:A + n]))
        rows.append((w["name"], float(err), float(g["nacc"].sum() / o["nacc"].sum())))
    for r in rows:
        print("FP32_RHS %s: max |end state - oracle| = %.3e, accepted steps vs oracle = %.3f" % r)
    # not a tolerance claim: a bound far above binary32 rounding that a wrong
    # forcing quadrant, sign or phase would exceed
    assert rows[0][1] < 1e-5


def test_fp32_rhs_forcing_phase_at_large_t():
    # the same Duffing sweep started 1000 forcing periods later: the binary32
    # forcing keeps the phase to binary32 rounding of a reduced angle, so the
    # error stays at the level of the run from t = 0 (a phase taken from t
    # rounded to binary32 would be off by up to 2.4e-4 rad here)
    w = W.duffing_rkck(16, 8, 4, 2)
    w = dict(w, td=w["td"] + 2000.0 * np.pi)
    o = run_oracle(w, NTHREADS)
    g = run_gpu(w, prec=G.ODE_FP32_RHS)
    A, n = DIMS[w["model"]][2], DIMS[w["model"]][0]
    err = np.max(np.abs(g["records"][:, A:A + n] - o["records"][:, A:A + n]))
    print("FP32_RHS duffing from t = 2000 pi: max |end state - oracle| = %.3e" % err)
    assert err < 1e-5


def test_fp32_rhs_full_size_sampled_report():
    """The binary32 form of the bench sweep at full size (2^17 systems, 1024 + 64
    periods): the error of sampled systems against the binary64 oracle is
    reported per quantity (no tolerance is claimed); a bound far above it
    guards against a broken form."""
    w = W.duffing_rkck()
    g = run_gpu(w, prec=G.ODE_FP32_RHS, autotune=True)
    assert np.all(g["status"] == 1)
    idx = W.sample_indices(w["N"], 256, corners=(0, 511, w["N"] - 512, w["N"] - 1))
    ws = W.subset(w, idx)
    mask, o = _nonchaotic(ws, w["n_transient"], w["n_record"], cont_rows=(4, 5, 7, 8), rtol=1e-10)
    rg, ro = g["records"][:, :, idx][:, :, mask], o["records"][:, :, mask]
    err = {name: float(np.max(np.abs(rg[:, row] - ro[:, row])))
           for name, row in (("event y1", 4), ("event t", 5), ("end y1", 7), ("end y2", 8))}
    _report("FP32_RHS duffing full size, %d of %d sampled points well-conditioned: %s" % (
        mask.sum(), len(idx), ", ".join("%s %.2e" % kv for kv in err.items())))
    assert mask.sum() >= 10 and max(err.values()) < 1e-3


def test_fp32_rhs_valve_full_size_sampled_report():
    """The binary32 form of the valve sweep at full size (2^16 systems, 1024 +
    64 iterations, Sec. 7.3): for 256 sampled systems, on the points where the
    binary64 oracle is well-conditioned (its rtol and rtol / 10 runs agree),
    the error against the oracle is reported per quantity -- the Poincare
    maximum y1 and its time, the state at the maximum, the impact count of
    each iteration and the stop status.  No tolerance is claimed; loose
    bounds guard against a broken form."""
    w = W.valve()
    s = gpu_solver(w, prec=G.ODE_FP32_RHS)
    try:
        gpu_load(s, w)
        G.ode_autotune(s, w["h0"], 2)
        rec = np.zeros((w["n_record"], 9, w["N"]))
        G.ode_run_periods(s, w["h0"], w["n_transient"], w["n_record"], rec)
        G.ode_synchronize(s)
        g = gpu_results(s, w, rec)
    finally:
        G.ode_destroy(s)
    idx = W.sample_indices(w["N"], 256, corners=(0, w["N"] // 2, w["N"] - 1))
    ws = W.subset(w, idx)
    stable, o = _valve_well_conditioned(ws, 100 * w["evt_tol"][0])
    rg, ro = g["records"][:, :, idx][:, :, stable], o["records"][:, :, stable]
    err = {}
    for name, row in (("Poincare max y1", 5), ("y2 at max", 6), ("y3 at max", 7)):
        d = np.abs(rg[:, row] - ro[:, row])
        err[name] = (float(np.median(d)), float(np.max(d)))
    # durations of the iterations (the absolute time drifts along the orbit)
    d = np.abs(np.diff(rg[:, 8], axis=0) - np.diff(ro[:, 8], axis=0))
    err["iteration duration"] = (float(np.median(d)), float(np.max(d)))
    imp_equal = float(np.mean(rg[:, 4] == ro[:, 4]))
    st_equal = float(np.mean(g["status"][idx][stable] == o["status"][stable]))
    _report("FP32_RHS valve full size, %d of %d sampled points well-conditioned: %s; impact counts equal "
            "in %.4f of iterations; status equal in %.4f of systems; accepted steps vs oracle %.3f" % (
                stable.sum(), len(idx), ", ".join("%s median %.2e max %.2e" % (k, a, b) for k, (a, b) in err.items()),
                imp_equal, st_equal, g["nacc"][idx].sum() / o["nacc"].sum()))
    assert stable.sum() >= 160
    assert np.all(np.isfinite(rg))
    assert err["Poincare max y1"][0] < 1e-3 and imp_equal > 0.9


# ---------------------------------------------------------------------------
# Edge cases: partial warps / blocks, a single system, empty and ragged time
# domains, NaN parameters, step budget.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 31, 33, 1025])
def test_ragged_sizes(N):
    w = W.duffing_rkck(N, 1, 2, 2)
    g = run_gpu(w)
    o = run_oracle(w, NTHREADS)
    assert np.all(g["status"] == 1)
    assert np.all(_rel_close(g["records"][:, 7:9], o["records"][:, 7:9], 1e-8, 1e-8))


def test_empty_and_mixed_time_domains():
    w = W.duffing_rkck(8, 1, 0, 2)
    td = w["td"].copy()
    td[1, 0] = 0.0          # empty domain: nothing to integrate
    td[1, 1] = -1.0         # reversed: treated as empty
    td[1, 2] = 1e-3         # shorter than h0
    td[:, 3] = [5.0, 7.5]   # shifted
    w = dict(w, td=td)
    g = run_gpu(w)
    o = run_oracle(w, NTHREADS)
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["nacc"][:2], 0)
    assert np.all(_rel_close(g["y"], o["y"], 1e-8, 1e-8))
    np.testing.assert_array_equal(g["records"][:, 9], o["records"][:, 9])


def test_nan_parameter_stops_at_hmin_and_budget():
    w = W.duffing_rkck(4, 1, 0, 1)
    p = w["p"].copy()
    p[0, 1] = float("nan")
    w = dict(w, p=p, hmin=1e-6)
    g = run_gpu(w)
    o = run_oracle(w, NTHREADS)
    np.testing.assert_array_equal(g["status"], o["status"])
    assert g["status"][1] == G.ODE_ST_HMIN_NAN
    np.testing.assert_array_equal(g["nrej"], o["nrej"])
    np.testing.assert_array_equal(g["y"][:, 1], w["y0"][:, 1])
    # step budget
    s = gpu_solver(dict(w, p=w["p"]))
    try:
        gpu_load(s, w)
        G.ode_set_step_budget(s, 7)
        G.ode_solve(s, w["h0"])
        G.ode_synchronize(s)
        r = gpu_results(s, w)
        ok = np.arange(w["N"]) != 1  # system 1 (NaN) stops at hmin first
        assert np.all(r["status"][ok] == G.ODE_ST_STEP_BUDGET)
        assert np.all(r["nacc"][ok] + r["nrej"][ok] == 7)
        assert r["status"][1] == G.ODE_ST_HMIN_NAN
    finally:
        G.ode_destroy(s)


# ---------------------------------------------------------------------------
# Object filling / read-back (Sec. 6.3, 6.10) and device pointers.
# ---------------------------------------------------------------------------
def test_linear_and_random_set_get_host_and_device():
    import torch
    w = W.duffing_rkck(16, 1, 0, 1)
    N = w["N"]
    s = gpu_solver(w)
    try:
        pool = 40
        td = np.arange(2 * pool, dtype=np.float64).reshape(2, pool)
        y = np.arange(2 * pool, dtype=np.float64).reshape(2, pool) + 1000
        p = np.arange(2 * pool, dtype=np.float64).reshape(2, pool) + 2000
        acc = np.arange(7 * pool, dtype=np.float64).reshape(7, pool) + 3000
        G.ode_linear_set(s, 2, 5, pool, 10, td=td, y=y, p=p, acc=acc)
        out = [np.zeros((c, N)) for c in (2, 2, 2, 7)]
        G.ode_linear_get(s, 0, 0, N, N, *out)
        for got, src in zip(out, (td, y, p, acc)):
            np.testing.assert_array_equal(got[:, 2:12], src[:, 5:15])
        io = np.array([15, 0, 7], dtype=np.int32)
        ip = np.array([1, 39, 20], dtype=np.int32)
        G.ode_random_set(s, io, ip, pool, 3, p=p, copy_mode=G.ODE_PARAM)
        pp = np.zeros((2, N))
        G.ode_linear_get(s, 0, 0, N, N, p=pp, copy_mode=G.ODE_PARAM)
        np.testing.assert_array_equal(pp[:, io], p[:, ip])
        # device pointers (torch tensors)
        dp = torch.tensor(p, device="cuda")
        dio, dip = torch.tensor(io, device="cuda"), torch.tensor(ip, device="cuda")
        G.ode_random_set(s, dio, dip, pool, 3, p=dp * 2, copy_mode=G.ODE_PARAM)
        torch.cuda.synchronize()
        back = torch.zeros((2, pool), dtype=torch.float64, device="cuda")
        G.ode_random_get(s, dio, dip, pool, 3, p=back, copy_mode=G.ODE_PARAM)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(back.cpu().numpy()[:, ip], 2 * p[:, ip])
        # invalid ranges are rejected with a message
        with pytest.raises(G.ODEError) as e:
            G.ode_linear_set(s, N - 1, 0, pool, 2, td=td, copy_mode=G.ODE_TIMEDOMAIN)
        assert "range" in str(e.value)
    finally:
        G.ode_destroy(s)


def test_device_records_and_single_solve_match_run_periods():
    import torch
    w = W.duffing_rkck(8, 2, 0, 3)
    N, A, n = w["N"], 7, 2
    ref = run_gpu(w)
    s = gpu_solver(w)
    try:
        gpu_load(s, w)
        rec = torch.zeros((3, A + n + 1, N), dtype=torch.float64, device="cuda")
        G.ode_run_periods(s, w["h0"], 0, 3, rec, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(rec.cpu().numpy(), ref["records"])
        # three single Solve calls give the same end state
        gpu_load(s, w)
        for _ in range(3):
            G.ode_solve(s, w["h0"])
        G.ode_synchronize(s)
        r = gpu_results(s, w)
        np.testing.assert_array_equal(r["y"], ref["y"])
    finally:
        G.ode_destroy(s)


def test_invalid_arguments_are_reported():
    with pytest.raises(G.ODEError):
        G.ode_create(7, 0, 0, 10, 0)
    with pytest.raises(G.ODEError) as e:
        G.ode_create(G.ODE_KELLER_MIKSIS, G.ODE_RKCK45, G.ODE_FP32_RHS, 10, 0)
    assert "binary64" in str(e.value)
    s = G.ode_create(G.ODE_DUFFING, G.ODE_RKCK45, G.ODE_FP64, 4, 0)
    try:
        with pytest.raises(G.ODEError):
            G.ode_set_tolerances(s, [1e-9, 1e-9], [1e-9, 1e-9], 1.0, 2.0, 5.0, 0.1)
        with pytest.raises(G.ODEError):
            G.ode_set_launch(s, 48, 0)
        with pytest.raises(G.ODEError):
            G.ode_set_launch(s, 64, 3)
        with pytest.raises(G.ODEError):
            G.ode_solve(s, -1.0)
        with pytest.raises(G.ODEError):
            G.ode_set_events(s, 1, [2], [1e-6], [0], 0)
    finally:
        G.ode_destroy(s)


def test_watchdog_stops_a_launch_that_runs_too_long():
    """Failure detection without a fault: a launch whose threads exceed the
    time limit stop their systems (status TIMEOUT) and the next synchronizing
    call reports ODE_ERR_TIMEOUT; the context stays usable."""
    w = W.duffing_rkck(64, 4, 0, 400)
    for persistent in (0, 1):
        s = gpu_solver(w, persistent=persistent)
        try:
            gpu_load(s, w)
            G.ode_set_time_limit(s, 1e-3)
            G.ode_run_periods(s, w["h0"], 0, 400, None)
            with pytest.raises(G.ODEError) as e:
                G.ode_synchronize(s)
            assert e.value.code == G.ODE_ERR_TIMEOUT
            status = np.zeros(w["N"], dtype=np.int32)
            G.ode_get_status(s, status)
            assert np.any(status == G.ODE_ST_TIMEOUT)
            # the solver and the context still work
            G.ode_set_time_limit(s, 300.0)
            gpu_load(s, w)
            G.ode_run_periods(s, w["h0"], 0, 1, None)
            G.ode_synchronize(s)
            G.ode_get_status(s, status)
            assert np.all(status == G.ODE_ST_TEND)
        finally:
            G.ode_destroy(s)


def test_autotune_restores_state_and_keeps_results():
    w = W.duffing_rkck(32, 4, 2, 2)
    ref = run_gpu(w)
    s = gpu_solver(w)
    try:
        gpu_load(s, w)
        t = G.ode_autotune(s, w["h0"], 2, full=True)
        assert t["block"] in (64, 96, 128, 160, 192, 256) and t["persistent"] in (0, 1, 2)
        assert t["systems_per_thread"] in (1, 2) and t["slices_per_launch"] in (0, 1) and t["warp_sync"] in (0, 1)
        trials = t["trial_ms"]
        assert trials.shape == (4, 6)
        assert np.all(trials[trials >= 0] > 0) and trials.max() > 0
        assert t["split_ms"][0] > 0 and t["split_ms"][2] == trials[trials >= 0].min()
        # every form that ran was also tried with warp-synchronous slices, and
        # the choice is the fastest trial of all
        ran = (trials >= 0).any(axis=1)
        assert np.all(t["warp_sync_ms"][ran] > 0) and np.all(t["warp_sync_ms"][~ran] == -1)
        allms = np.concatenate([trials[trials >= 0], t["split_ms"][t["split_ms"] >= 0],
                                t["warp_sync_ms"][t["warp_sync_ms"] >= 0]])
        form = {(0, 1): 0, (0, 2): 1, (1, 1): 2, (2, 1): 3}[(t["persistent"], t["systems_per_thread"])]
        if t["warp_sync"]:
            chosen = t["warp_sync_ms"][form]
        elif t["slices_per_launch"] == 1:
            chosen = t["split_ms"][0]
        elif t["slices_per_launch"] > 1:
            chosen = t["split_ms"][1]
        else:
            chosen = trials[form][[64, 96, 128, 160, 192, 256].index(t["block"])]
        assert chosen == allms.min()
        rec = np.zeros((2, 10, w["N"]))
        G.ode_run_periods(s, w["h0"], 2, 2, rec)
        G.ode_synchronize(s)
        r = gpu_results(s, w, rec)
        for key in ("records", "y", "acc", "nacc", "status"):
            np.testing.assert_array_equal(r[key], ref[key])
    finally:
        G.ode_destroy(s)


def test_persistent_refill_beyond_the_first_wave_is_identical():
    """More systems than the persistent grid has threads (2^17 Duffing systems,
    64-thread blocks: one wave of 77 824 threads on 152 SMs), so the device
    queue hands out the systems after the first wave in both orders, with and
    without warp-synchronous slices: records, end states, step counts and
    statuses are bitwise those of the per-sweep launch (every system is run
    exactly once, whoever runs it)."""
    w = W.duffing_rkck(n_transient=1, n_record=2)
    ref = run_gpu(w, block=64)
    for pers in (1, 2):
        for ws in (0, 1):
            s = gpu_solver(w, block=64, persistent=pers)
            try:
                assert G.ode_kernel_info(w["model"], w["scheme"], G.ODE_FP64, 1, 64)["blocks_per_sm"] * 152 * 64 < w["N"]
                G.ode_set_schedule(s, 1, 0, ws)
                gpu_load(s, w)
                rec = np.zeros((w["n_record"], 10, w["N"]))
                G.ode_run_periods(s, w["h0"], w["n_transient"], w["n_record"], rec)
                G.ode_synchronize(s)
                r = gpu_results(s, w, rec)
            finally:
                G.ode_destroy(s)
            for key in ("records", "y", "acc", "nacc", "status"):
                np.testing.assert_array_equal(r[key], ref[key], err_msg="%s pers %d ws %d" % (key, pers, ws))


@pytest.mark.parametrize("spt,spl,ws,pers", [(2, 0, 0, 0), (3, 1, 0, 0), (1, 2, 1, 0), (5, 3, 1, 0),
                                             (1, 0, 1, 0), (1, 0, 1, 1), (1, 2, 1, 2)])
def test_schedule_leaves_results_unchanged(spt, spl, ws, pers):
    """Several systems per thread (per-sweep launch), runs split into launches
    of a few slices and warp-synchronous slices give bitwise the same
    records, states, counters and statuses as one system per thread in one
    launch; 333 systems leave a ragged last block."""
    for w in (W.duffing_rkck(37, 9, 3, 2), W.valve(N=333, n_transient=3, n_record=2)):
        ref = run_gpu(w)
        n, P, A, E = DIMS[w["model"]]
        s = gpu_solver(w, block=64, persistent=pers)
        try:
            G.ode_set_schedule(s, spt, spl, ws)
            gpu_load(s, w)
            rec = np.zeros((w["n_record"], A + n + 1, w["N"]))
            G.ode_run_periods(s, w["h0"], w["n_transient"], w["n_record"], rec)
            G.ode_synchronize(s)
            r = gpu_results(s, w, rec)
        finally:
            G.ode_destroy(s)
        for key in ("records", "y", "acc", "td", "nacc", "nrej", "status", "ecnt"):
            np.testing.assert_array_equal(r[key], ref[key], err_msg=key)


def test_kernels_do_not_spill():
    """Every integrator kernel launches (at least one resident block per SM)
    and keeps its state in registers: its local memory is at most the 40-byte
    call frame of the out-of-line event-root prediction, with no room for
    spilled registers beyond it."""
    for model in (0, 1, 2, 3, 4):
        for scheme in (0, 1):
            for prec in ((0, 1) if model in (0, 2, 3) else (0,)):
                for pers in (0, 1):
                    info = G.ode_kernel_info(model, scheme, prec, pers)
                    assert info["blocks_per_sm"] >= 1
                    assert info["regs"] <= 255
                    assert info["local_bytes"] <= 40, (model, scheme, prec, pers, info)


@pytest.mark.parametrize("case", ["second_not_crossed_at_located_point", "second_crossed_before_it"])
def test_valve_two_events_in_one_step_parity(case):
    """Both event surfaces crossed within one fixed step of size 1 (Sec. 4):
    only the impact (highest index) is located; the other event fires at the
    located point only if it is crossed there.  Event counts, accessories and
    the end state equal the oracle's (the oracle pins this rule by brute
    force)."""
    direction, y0, delta = {"second_not_crossed_at_located_point": ((1, -1), [0.01, -1.0, 1.0], 0.5),
                            "second_crossed_before_it": ((-1, -1), [0.05, 0.1, 1.0], 2.0)}[case]
    N = 4  # the same system four times: one partial warp
    p = np.tile(np.array([[1.25], [delta], [0.1], [1.0], [0.8]]), (1, N))
    w = dict(W.valve(N=N, n_transient=0, n_record=1), p=p, rtol=1e-6, atol=1e-6, hmin=1.0, hmax=1.0,
             h0=1.0, evt_dir=direction, evt_tol=(1e-10, 1e-10), evt_stop=(0, 0), max_eq=0, td_mode=W.TD_KEEP,
             td=np.vstack([np.zeros(N), np.full(N, 3.0)]), y0=np.tile(np.array(y0)[:, None], (1, N)))
    g = run_gpu(w)
    o = run_oracle(w, 1)
    np.testing.assert_array_equal(g["ecnt"], o["ecnt"])
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["acc"][4], o["acc"][4])  # impacts
    np.testing.assert_allclose(g["y"], o["y"], rtol=1e-8, atol=1e-8)


# ---------------------------------------------------------------------------
# Chaotic parameter points (Sec. 7.1.1): no pointwise agreement is possible
# beyond a short horizon, so the acceptance is (a) agreement over the first
# periods from the initial conditions and (b) Poincare-section statistics.
# ---------------------------------------------------------------------------
def _gpu_records_sampled(w, idx, n_tr, n_rec, autotune=True):
    """Run the whole sweep w with device-resident records (the bench's launch
    form, autotuned) and return the records of systems idx only."""
    import torch
    n, P, A, E = DIMS[w["model"]]
    s = gpu_solver(w)
    try:
        gpu_load(s, w)
        if autotune:
            G.ode_autotune(s, w["h0"], 4)
        rec = torch.zeros((n_rec, A + n + 1, w["N"]), dtype=torch.float64, device="cuda")
        G.ode_run_periods(s, w["h0"], n_tr, n_rec, rec)
        G.ode_synchronize(s)
        st = np.zeros(w["N"], dtype=np.int32)
        G.ode_get_status(s, st)
        sel = torch.as_tensor(np.asarray(idx), device="cuda")
        return rec.index_select(2, sel).cpu().numpy(), st
    finally:
        G.ode_destroy(s)


def _distinct(a, digits=6):
    return len(np.unique(np.round(a, digits)))


def _section_statistics(A, B, cols):
    """Per-system two-sample KS p-values of Poincare sets A[:, i], B[:, i],
    the median |difference of means|, the median |log variance ratio| and the
    KS distance between the pooled sets."""
    from scipy.stats import ks_2samp
    p = np.array([ks_2samp(A[:, i], B[:, i]).pvalue for i in cols])
    dm = np.median([abs(A[:, i].mean() - B[:, i].mean()) for i in cols])
    lv = np.median([abs(math.log(A[:, i].var() / B[:, i].var())) for i in cols])
    pooled = ks_2samp(A[:, cols].ravel(), B[:, cols].ravel()).statistic
    return dict(reject=float((p < 0.01).mean()), dmean=float(dm), dlogvar=float(lv), pooled_ks=float(pooled))


def test_duffing_chaotic_points_short_horizon_and_poincare_statistics():
    """The paper's double-well Duffing (delta = +1, Sec. 7.1.1) on the bench's
    full grid (512 x 256, k in [0.2, 0.3], B in [0.3, 0.5], 2^17 systems,
    RKCK45 rtol 1e-10, maxima located to 1e-12) in the bench's launch form.
    Most of these points are chaotic.  512 sampled systems are replayed by
    the oracle:
      (a) from the initial conditions, the first three periods agree within
          100 x rtol on every sampled point (records: located maximum and its
          time, Poincare point);
      (b) after 64 transient periods, the Poincare sets y1(2 pi n) of 256
          recorded periods on the chaotic points (more than 32 distinct
          values) are compared GPU against oracle with the two-sample KS test
          at alpha = 0.01, the means and the variances.  Serial correlation
          makes the nominal 1 % rejection rate meaningless, so the reference
          is the oracle against itself with atol perturbed by 1e-3 relative (a
          perturbation at the scale of rounding): the GPU's rejection rate may
          exceed it by at most 0.05, its median |mean difference| and
          |log variance ratio| may be at most twice the oracle's, and so may
          the KS distance between the pooled sets of all chaotic points
          (pooled, the sets are too correlated for a nominal KS level)."""
    w = dict(W.duffing_rkck(), mc=(1.0, 1.0, 1.0), name="duffing_double_well_512x256")
    idx = W.sample_indices(w["N"], 512, corners=(0, 511, w["N"] - 512, w["N"] - 1))
    ws = W.subset(w, idx)
    # (a) short horizon
    g, st = _gpu_records_sampled(w, idx, 0, 3)
    assert np.all(st == 1)
    o = run_oracle(ws, NTHREADS, n_transient=0, n_record=3)["records"]
    tol = 100 * 1e-10
    for row in (4, 5, 7, 8):
        assert np.all(np.abs(g[:, row] - o[:, row]) <= tol * (1 + np.abs(o[:, row]))), row
    np.testing.assert_array_equal(g[:, 6], o[:, 6])  # maxima per period
    # (b) Poincare statistics after the transient
    n_tr, n_rec = 64, 256
    g, st = _gpu_records_sampled(w, idx, n_tr, n_rec)
    assert np.all(st == 1)
    o1 = run_oracle(ws, NTHREADS, n_transient=n_tr, n_record=n_rec)["records"]
    o2 = run_oracle(ws, NTHREADS, n_transient=n_tr, n_record=n_rec, atol=1.001e-10)["records"]
    Pg, P1, P2 = g[:, 7], o1[:, 7], o2[:, 7]
    chaotic = np.array([i for i in range(len(idx)) if _distinct(P1[:, i]) > 32])
    assert len(chaotic) >= 128
    gpu = _section_statistics(Pg, P1, chaotic)
    ref = _section_statistics(P2, P1, chaotic)
    _report("duffing double well full grid: %d of %d sampled points chaotic; GPU vs oracle %s; "
            "oracle vs perturbed oracle %s" % (len(chaotic), len(idx), gpu, ref))
    assert gpu["reject"] <= ref["reject"] + 0.05
    assert gpu["dmean"] <= 2 * ref["dmean"] and gpu["dlogvar"] <= 2 * ref["dlogvar"]
    assert gpu["pooled_ks"] <= 2 * ref["pooled_ks"] + 0.01
    # the attractor's range is the same: every GPU section point lies within
    # the oracle's envelope over all chaotic points, widened by 1 %
    lo, hi = P1[:, chaotic].min(), P1[:, chaotic].max()
    assert Pg[:, chaotic].min() >= lo - 0.01 * (hi - lo) and Pg[:, chaotic].max() <= hi + 0.01 * (hi - lo)


def test_duffing_bench_grid_conditioning_census():
    """Every system of the bench sweep (hardening Duffing, 2^17 systems, 1024 +
    64 periods) integrated on the GPU at rtol and at rtol / 10: the fraction
    whose records agree within 10 x rtol (the well-conditioned criterion) is
    reported.  Up to 64 of the systems that disagree are replayed by the
    oracle, which must find them ill-conditioned too (its own rtol and
    rtol / 10 runs disagree as well), or agree with the GPU at 100 x rtol."""
    import torch
    w = W.duffing_rkck()
    recs = []
    for rt in (1e-10, 1e-11):
        ww = dict(w, rtol=rt, atol=rt)
        s = gpu_solver(ww)
        try:
            gpu_load(s, ww)
            rec = torch.zeros((w["n_record"], 10, w["N"]), dtype=torch.float64, device="cuda")
            G.ode_run_periods(s, w["h0"], w["n_transient"], w["n_record"], rec)
            G.ode_synchronize(s)
            recs.append(rec)
        finally:
            G.ode_destroy(s)
    a, b = recs[0][:, [4, 5, 7, 8]], recs[1][:, [4, 5, 7, 8]]
    ok = ((a - b).abs() <= 1e-9 * (1 + b.abs())).all(dim=1).all(dim=0).cpu().numpy()
    bad = np.where(~ok)[0]
    _report("duffing_rkck bench grid: %d of %d systems well-conditioned on the GPU (rtol vs rtol/10)"
            % (ok.sum(), w["N"]))
    assert ok.mean() > 0.9
    if len(bad):
        pick = bad[np.linspace(0, len(bad) - 1, min(64, len(bad))).astype(int)]
        ws = W.subset(w, pick)
        mask, o = _nonchaotic(ws, w["n_transient"], w["n_record"], cont_rows=(4, 5, 7, 8), rtol=1e-10)
        g = recs[0][:, :, torch.as_tensor(pick, device="cuda")].cpu().numpy()
        agree = np.all(np.abs(g[:, [4, 5, 7, 8]] - o["records"][:, [4, 5, 7, 8]])
                       <= 1e-8 * (1 + np.abs(o["records"][:, [4, 5, 7, 8]])), axis=(0, 1))
        _report("  of %d replayed: %d ill-conditioned for the oracle too, %d agree with it at 100 x rtol"
                % (len(pick), (~mask).sum(), agree.sum()))
        assert np.all(~mask | agree)
