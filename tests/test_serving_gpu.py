"""Serving (continuous batching): a request's results are the same alone and
in a mix of requests of other models, sizes and horizons that arrive while it
is resident, and equal to a plain ode_run_periods of the same systems."""
import time

import numpy as np
import pytest

import workloads as W
from paper_1810_03931_gb300 import odegpu as G
from paper_1810_03931_gb300.sweeps import settings_for

from _runners import DIMS, km_params_gpu, run_gpu

pytestmark = pytest.mark.gpu


def make_server(slice_periods=3):
    srv = G.ode_server_create(0, 1 << 30, slice_periods)
    G.ode_server_add_model(srv, settings_for(W.duffing_rkck(1, 1, 0, 1)), 1e-2, 4096)
    G.ode_server_add_model(srv, settings_for(W.valve(1, 0, 1)), 1e-2, 4096)
    G.ode_server_add_model(srv, settings_for(W.keller_miksis(1, 1, 0, 1)), 1e-2, 4096)
    G.ode_server_add_model(srv, settings_for(W.duffing_lyapunov(1, 0, 1)), 1e-2, 1024)
    return srv


def request(model, n, periods, seed):
    w = W.request_inputs(dict(model=model, size=n, horizon=periods, seed=seed))
    p = km_params_gpu(w) if model == W.KELLER_MIKSIS else w["p"]
    return w, p


def drain(srv, tickets, timeout=120.0):
    t0 = time.time()
    done = {}
    while len(done) < len(tickets):
        G.ode_server_progress(srv)
        for t, (model, n) in tickets.items():
            if t not in done and G.ode_server_poll(srv, t) == 2:
                nsys, _, A, _ = DIMS[model]
                done[t] = G.ode_server_result(srv, t, n, nsys, A)
        assert time.time() - t0 < timeout
        time.sleep(0.0005)
    return done


def test_request_alone_and_in_the_mix_are_identical():
    wa, pa = request(W.DUFFING, 150, 7, seed=11)
    srv = make_server()
    try:
        ta = G.ode_server_submit(srv, W.DUFFING, 7, wa["td"], wa["y0"], pa)
        alone = drain(srv, {ta: (W.DUFFING, 150)})[ta]
    finally:
        G.ode_server_destroy(srv)
    srv = make_server()
    try:
        tickets = {}
        others = [(W.KELLER_MIKSIS, 40, 5, 1), (W.VALVE, 300, 4, 2), (W.DUFFING, 1000, 5, 3),
                  (W.DUFFING, 3000, 2, 4), (W.VALVE, 77, 9, 5)]
        for k, (m, n, h, sd) in enumerate(others):
            w, p = request(m, n, h, sd)
            tickets[G.ode_server_submit(srv, m, h, w["td"], w["y0"], p)] = (m, n)
            if k == 2:  # the request arrives while others are resident
                for _ in range(5):
                    G.ode_server_progress(srv)
                ta2 = G.ode_server_submit(srv, W.DUFFING, 7, wa["td"], wa["y0"], pa)
                tickets[ta2] = (W.DUFFING, 150)
        res = drain(srv, tickets)
        mixed = res[ta2]
    finally:
        G.ode_server_destroy(srv)
    for key in ("td", "y", "acc", "status", "nacc"):
        np.testing.assert_array_equal(alone[key], mixed[key], err_msg=key)
    # and the same as a plain iterated integration of those systems
    w = dict(wa, p=pa, n_transient=6, n_record=1)
    ref = run_gpu(w, persistent=1)
    np.testing.assert_array_equal(mixed["y"], ref["y"])
    np.testing.assert_array_equal(mixed["acc"], ref["acc"])
    np.testing.assert_array_equal(mixed["nacc"], ref["nacc"])
    assert mixed["latency"] > 0


def test_admission_waits_for_slots_and_rejects_oversized_requests():
    srv = G.ode_server_create(0, 1 << 30, 2)
    try:
        G.ode_server_add_model(srv, settings_for(W.duffing_rkck(1, 1, 0, 1)), 1e-2, 256)
        w, p = request(W.DUFFING, 200, 3, 7)
        t1 = G.ode_server_submit(srv, W.DUFFING, 3, w["td"], w["y0"], p)
        t2 = G.ode_server_submit(srv, W.DUFFING, 3, w["td"], w["y0"], p)
        G.ode_server_progress(srv)
        # only one 200-system request fits in 256 slots: the other waits
        assert G.ode_server_poll(srv, t1) == 1 and G.ode_server_poll(srv, t2) == 0
        res = drain(srv, {t1: (W.DUFFING, 200), t2: (W.DUFFING, 200)})
        for key in ("y", "acc", "nacc"):
            np.testing.assert_array_equal(res[t1][key], res[t2][key])
        big, pb = request(W.DUFFING, 300, 1, 8)
        with pytest.raises(G.ODEError):
            G.ode_server_submit(srv, W.DUFFING, 1, big["td"], big["y0"], pb)
        with pytest.raises(G.ODEError):  # pool beyond the HBM budget
            G.ode_server_add_model(srv, settings_for(W.valve(1, 0, 1)), 1e-2, 1 << 30)
    finally:
        G.ode_server_destroy(srv)


def test_tuned_chunk_length_and_a_lyapunov_pool():
    """Chunk length tuned per request (slice_periods = 0) gives the same
    results as fixed chunks; the Lyapunov model is served like the others."""
    wa, pa = request(W.DUFFING, 300, 9, seed=21)
    wl = W.duffing_lyapunov(N=100, n_transient=4, n_record=1)
    out = {}
    for sp in (0, 2):
        srv = make_server(slice_periods=sp)
        try:
            ta = G.ode_server_submit(srv, W.DUFFING, 9, wa["td"], wa["y0"], pa)
            tl = G.ode_server_submit(srv, W.DUFFING_LYAPUNOV, 5, wl["td"], wl["y0"], wl["p"])
            out[sp] = drain(srv, {ta: (W.DUFFING, 300), tl: (W.DUFFING_LYAPUNOV, 100)})
            out[sp] = (out[sp][ta], out[sp][tl])
        finally:
            G.ode_server_destroy(srv)
    for i in range(2):
        for key in ("td", "y", "acc", "status", "nacc"):
            np.testing.assert_array_equal(out[0][i][key], out[2][i][key], err_msg=key)
    ref = run_gpu(wl, persistent=0)
    np.testing.assert_array_equal(out[0][1]["y"], ref["y"])
    np.testing.assert_array_equal(out[0][1]["acc"], ref["acc"])


def test_reused_slot_range_with_distinct_requests_matches_oracle():
    """A pool of 256 slots and three 200-system requests with distinct seeds:
    each request reuses the range the previous one held (it may be admitted on
    another stream while the previous results are still being copied out).
    Each request's end state and accessories are checked bitwise against a
    plain ode_run_periods of the same systems and against the CPU oracle
    (100 x rtol on well-conditioned points, counts exact)."""
    from _runners import run_oracle
    from test_parity_gpu import NTHREADS, _nonchaotic

    horizon = 4
    srv = G.ode_server_create(0, 1 << 30, 1)
    reqs = {}
    try:
        G.ode_server_add_model(srv, settings_for(W.duffing_rkck(1, 1, 0, 1)), 1e-2, 256)
        for sd in (31, 32, 33):
            w, p = request(W.DUFFING, 200, horizon, sd)
            reqs[G.ode_server_submit(srv, W.DUFFING, horizon, w["td"], w["y0"], p)] = w
        G.ode_server_progress(srv)
        states = [G.ode_server_poll(srv, t) for t in reqs]
        assert states.count(1) == 1 and states.count(0) == 2  # one range, one request at a time
        res = drain(srv, {t: (W.DUFFING, 200) for t in reqs})
    finally:
        G.ode_server_destroy(srv)
    for t, w in reqs.items():
        got = res[t]
        ww = dict(w, n_transient=horizon - 1, n_record=1)
        ref = run_gpu(ww, persistent=0)
        for key in ("td", "y", "acc", "status", "nacc"):
            np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
        mask, o = _nonchaotic(ww, horizon - 1, 1, cont_rows=(4, 5, 7, 8), rtol=1e-10)
        assert mask.sum() >= 150
        tol = 100 * 1e-10
        for m in range(2):
            assert np.all(np.abs(got["y"][m, mask] - o["y"][m, mask]) <= tol * (1 + np.abs(o["y"][m, mask])))
        for a in (4, 5):  # first located maximum of the last period and its time
            assert np.all(np.abs(got["acc"][a, mask] - o["acc"][a, mask])
                          <= tol * (1 + np.abs(o["acc"][a, mask])))
        np.testing.assert_array_equal(got["acc"][6, mask], o["acc"][6, mask])  # maxima counted
        np.testing.assert_array_equal(got["status"], o["status"])
        # the requests differ, so a late copy of a previous occupant would show
        assert not np.array_equal(got["y"], res[list(reqs)[0]]["y"]) or t == list(reqs)[0]


def test_late_small_request_overtakes_a_large_one():
    """Continuous batching in one launch: a large Duffing request (more
    systems than the serving kernel has threads) holds the GPU; a small request
    submitted afterwards gets threads as soon as systems are handed back (a
    residency quantum of 4 periods) and finishes long before the large one,
    whose results are unchanged (bitwise equal to a plain integration of a
    sample of its systems)."""
    srv = G.ode_server_create(0, 8 << 30, 4)
    try:
        G.ode_server_add_model(srv, settings_for(W.duffing_rkck(1, 1, 0, 1)), 1e-2, 1 << 17)
        wb, pb = request(W.DUFFING, 100000, 24, 101)
        ws, ps = request(W.DUFFING, 10, 2, 102)
        tb = G.ode_server_submit(srv, W.DUFFING, 24, wb["td"], wb["y0"], pb)
        t0 = time.time()
        while time.time() - t0 < 0.3:  # the large request is running
            G.ode_server_progress(srv)
            time.sleep(0.0005)
        ts = G.ode_server_submit(srv, W.DUFFING, 2, ws["td"], ws["y0"], ps)
        res = drain(srv, {tb: (W.DUFFING, 100000), ts: (W.DUFFING, 10)}, timeout=300)
        st = G.ode_server_stats(srv, W.DUFFING)
    finally:
        G.ode_server_destroy(srv)
    assert res[ts]["latency"] < 0.5 * res[tb]["latency"], (res[ts]["latency"], res[tb]["latency"])
    assert st["yielded"] > 0 and st["flags"] == 0 and st["unfinished"] == 0
    idx = W.sample_indices(100000, 64)
    wsub = dict(W.subset(wb, idx), n_transient=23, n_record=1)
    wsub["p"] = np.ascontiguousarray(pb[:, idx])
    ref = run_gpu(wsub, persistent=0)
    for key in ("td", "y", "acc", "status", "nacc"):
        np.testing.assert_array_equal(res[tb][key][..., idx], ref[key], err_msg=key)
