"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against something the mathematics or the paper
fixes: order conditions of the published tableaux, closed-form solutions,
conservation laws, the restitution law, library integrators (scipy) on the
dimensional Keller-Miksis equation, and brute force on tiny cases.  They run
on the CPU (not marked gpu).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_settings.json")))


def _frac(x):
    return Fraction(x).limit_denominator(1 << 20)


# --------------------------------------------------------------------------
# Tableaux (Sec. 3): order conditions in exact rational arithmetic.
# --------------------------------------------------------------------------
def _order_conditions(A, b, c, order):
    """Residuals of the Butcher order conditions up to `order` (exact)."""
    s = len(b)
    dot = lambda u, v: sum(u[i] * v[i] for i in range(s))
    Av = lambda v: [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]
    mul = lambda u, v: [u[i] * v[i] for i in range(s)]
    one = [Fraction(1)] * s
    c2, c3, c4 = mul(c, c), mul(mul(c, c), c), mul(mul(c, c), mul(c, c))
    Ac, Ac2, Ac3 = Av(c), Av(c2), Av(c3)
    conds = [(dot(b, one), Fraction(1))]
    if order >= 2:
        conds += [(dot(b, c), Fraction(1, 2))]
    if order >= 3:
        conds += [(dot(b, c2), Fraction(1, 3)), (dot(b, Ac), Fraction(1, 6))]
    if order >= 4:
        conds += [(dot(b, c3), Fraction(1, 4)), (dot(b, mul(c, Ac)), Fraction(1, 8)),
                  (dot(b, Ac2), Fraction(1, 12)), (dot(b, Av(Ac)), Fraction(1, 24))]
    if order >= 5:
        conds += [(dot(b, c4), Fraction(1, 5)), (dot(b, mul(c2, Ac)), Fraction(1, 10)),
                  (dot(b, mul(c, Ac2)), Fraction(1, 15)), (dot(b, mul(c, Av(Ac))), Fraction(1, 30)),
                  (dot(b, mul(Ac, Ac)), Fraction(1, 20)), (dot(b, Ac3), Fraction(1, 20)),
                  (dot(b, Av(mul(c, Ac))), Fraction(1, 40)), (dot(b, Av(Ac2)), Fraction(1, 60)),
                  (dot(b, Av(Av(Ac))), Fraction(1, 120))]
    return [lhs - rhs for lhs, rhs in conds]


def test_cash_karp_order_conditions():
    c, a, b5, b4 = O.ck_tableau()
    A = [[_frac(a[i, j]) for j in range(6)] for i in range(6)]
    C = [_frac(x) for x in c]
    B5 = [_frac(x) for x in b5]
    B4 = [_frac(x) for x in b4]
    # consistency c_i = sum_j a_ij, explicit (strictly lower triangular)
    for i in range(6):
        assert sum(A[i]) == C[i]
        assert all(A[i][j] == 0 for j in range(i, 6))
    assert all(r == 0 for r in _order_conditions(A, B5, C, 5)), "fifth-order weights"
    assert all(r == 0 for r in _order_conditions(A, B4, C, 4)), "fourth-order weights"
    # the embedded pair is genuinely of different order
    assert any(r != 0 for r in _order_conditions(A, B4, C, 5))
    # the stored doubles are the nearest doubles to those rationals
    for x in list(c) + list(b5) + list(b4) + list(a.ravel()):
        f = _frac(x)
        assert float(f) == x


def test_rk4_order_conditions():
    c, a, b = O.rk4_tableau()
    A = [[_frac(a[i, j]) for j in range(4)] for i in range(4)]
    C = [_frac(x) for x in c]
    B = [_frac(x) for x in b]
    assert all(r == 0 for r in _order_conditions(A, B, C, 4))
    assert any(r != 0 for r in _order_conditions(A, B, C, 5))


# --------------------------------------------------------------------------
# Linear damped forced oscillator: x'' + k x' + x = B cos t (Duffing, c3 = 0).
# --------------------------------------------------------------------------
LIN_MC = (-1.0, 0.0, 1.0)


def linear_closed_form(t, x0, v0, k, B):
    """x, x' of x'' + k x' + x = B cos t (resonant forcing; x_p = B/k sin t)."""
    wd = np.sqrt(1.0 - k * k / 4.0)
    C1 = x0
    C2 = (v0 - B / k + k * x0 / 2.0) / wd
    e = np.exp(-k * t / 2.0)
    x = e * (C1 * np.cos(wd * t) + C2 * np.sin(wd * t)) + B / k * np.sin(t)
    v = (e * (-k / 2.0 * (C1 * np.cos(wd * t) + C2 * np.sin(wd * t))
              + (-C1 * wd * np.sin(wd * t) + C2 * wd * np.cos(wd * t))) + B / k * np.cos(t))
    return x, v


def _lin_inputs(N=5):
    k = np.linspace(0.2, 0.3, N)
    B = np.full(N, 0.3)
    td = np.vstack([np.zeros(N), np.full(N, 2 * math.pi)])
    y = np.vstack([np.full(N, -0.5), np.full(N, 0.1)])
    return k, B, td, y


def test_linear_oscillator_rkck_closed_form():
    k, B, td, y = _lin_inputs()
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=1e-12, atol=1e-12, mc=LIN_MC)
    n_per = 5
    r = O.run(cfg, td, y, np.vstack([k, B]), n_slices=n_per, record=True)
    assert np.all(r["status"] == O.ST_TEND)
    for s in range(n_per):
        x, v = linear_closed_form(2 * math.pi * (s + 1), -0.5, 0.1, k, B)
        rec = r["records"][s]
        A = 7
        np.testing.assert_allclose(rec[A + 0], x, rtol=0, atol=2e-10)
        np.testing.assert_allclose(rec[A + 1], v, rtol=0, atol=2e-10)
        np.testing.assert_allclose(rec[A + 2], 2 * math.pi, rtol=0, atol=0)


def test_linear_oscillator_rk4_error_bound():
    k, B, td, y = _lin_inputs()
    errs = []
    for nst in (250, 500, 1000):
        cfg = O.make_config(O.DUFFING, O.RK4, 2 * math.pi / nst, mc=LIN_MC)
        r = O.run(cfg, td, y, np.vstack([k, B]), n_slices=2)
        assert np.all(r["nacc"] == 2 * nst)
        x, v = linear_closed_form(4 * math.pi, -0.5, 0.1, k, B)
        errs.append(np.max(np.abs(r["y"][0] - x)))
    assert errs[-1] < 1e-9
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for q in ratios:
        assert 14.0 < q < 18.0, ratios


def test_linear_oscillator_maxima_times():
    """Event F = y2, direction -1 (local maxima of y1, Sec. 7.1.2) against the
    zeros of the closed-form velocity with negative acceleration."""
    from scipy.optimize import brentq
    kk, BB = 0.25, 0.3
    T = 6 * math.pi
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=1e-12, atol=1e-12, mc=LIN_MC,
                        events_on=True, evt_dir=(-1,), evt_tol=(1e-12,))
    tr = O.trace_slice(cfg, [0.0, T], [-0.5, 0.1], [kk, BB])
    vel = lambda t: linear_closed_form(t, -0.5, 0.1, kk, BB)[1]
    grid = np.linspace(0, T, 20001)
    vg = vel(grid)
    roots = [brentq(vel, grid[i], grid[i + 1], xtol=1e-15)
             for i in range(len(grid) - 1) if vg[i] > 0 >= vg[i + 1]]
    assert len(roots) == len(tr["ev_t"]) >= 2
    np.testing.assert_allclose(tr["ev_t"], roots, rtol=0, atol=1e-9)
    assert np.all(np.abs(tr["ev_y"][:, 1]) <= 1e-12)
    assert tr["ecnt"][0] == len(roots)


# --------------------------------------------------------------------------
# Observed order (Sec. 3): RK4 is fourth order, the propagated Cash-Karp
# solution fifth order; the embedded estimate is the fourth-order local error.
# --------------------------------------------------------------------------
def _duffing_reference(T, y0, k, B):
    from scipy.integrate import solve_ivp
    f = lambda t, y: [y[1], -y[0] - y[0] ** 3 - k * y[1] + B * math.cos(t)]
    s = solve_ivp(f, (0, T), y0, method="DOP853", rtol=1e-14, atol=1e-15)
    return s.y[:, -1]


@pytest.mark.parametrize("scheme,expected", [(O.RK4, 16.0), (O.RKCK45, 32.0)])
def test_observed_global_order(scheme, expected):
    T, y0, k, B = 2.0, [-0.5, 0.1], 0.25, 0.3
    ref = _duffing_reference(T, y0, k, B)
    errs = []
    for h in (0.1, 0.05, 0.025):
        if scheme == O.RK4:
            cfg = O.make_config(O.DUFFING, O.RK4, h)
        else:  # fixed step: hmin = hmax = h accepts every step
            cfg = O.make_config(O.DUFFING, O.RKCK45, h, hmin=h, hmax=h)
        r = O.run(cfg, [[0.0], [T]], [[y0[0]], [y0[1]]], [[k], [B]])
        assert int(r["nacc"][0]) == round(T / h)
        errs.append(np.max(np.abs(r["y"][:, 0] - ref)))
    for i in range(2):
        q = errs[i] / errs[i + 1]
        assert 0.8 * expected < q < 1.25 * expected, (errs, q)


def test_embedded_estimate_is_fourth_order_local_error():
    y0, k, B = np.array([-0.5, 0.1]), 0.25, 0.3
    cfg = O.make_config(O.DUFFING, O.RKCK45, 0.1)
    prev = None
    for h in (0.1, 0.05, 0.025):
        y5, e = O.single_step(cfg, 0.0, y0, [k, B], h)
        ref = _duffing_reference(h, list(y0), k, B)
        y4 = y5 - e
        # the propagated solution is more accurate than the embedded one
        assert np.max(np.abs(y5 - ref)) < 0.2 * np.max(np.abs(e))
        # and the estimate tracks the true fourth-order local error
        assert np.max(np.abs((y4 - ref) + e)) < 0.2 * np.max(np.abs(e))
        if prev is not None:
            q = np.max(np.abs(prev)) / np.max(np.abs(e))
            assert 24 < q < 40
        prev = e


# --------------------------------------------------------------------------
# Conservation: undamped, unforced Duffing keeps E = y2^2/2 - d y1^2/2 + c y1^4/4.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [-1.0, 1.0])
def test_duffing_energy_conservation(delta):
    N = 4
    y = np.vstack([np.linspace(-1.2, 1.5, N), np.linspace(0.3, -0.2, N)])
    E0 = y[1] ** 2 / 2 - delta * y[0] ** 2 / 2 + y[0] ** 4 / 4
    p = np.zeros((2, N))
    drifts = []
    for rtol in (1e-8, 1e-10, 1e-12):
        cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=rtol, atol=rtol, mc=(delta, 1.0, 1.0))
        r = O.run(cfg, [np.zeros(N), np.full(N, 50.0)], y, p)
        E1 = r["y"][1] ** 2 / 2 - delta * r["y"][0] ** 2 / 2 + r["y"][0] ** 4 / 4
        drifts.append(np.max(np.abs(E1 - E0)))
        assert drifts[-1] < 1000 * rtol
    assert drifts[0] > drifts[1] > drifts[2]


# --------------------------------------------------------------------------
# Impact law (Eqs. (32)-(34)) on a bouncing ball: polynomial free flight is
# integrated exactly, so impact times and velocities follow in closed form.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", [O.RK4, O.RKCK45])
def test_bouncing_ball_restitution(scheme):
    g, r_, h0 = 1.0, 0.8, 1.0
    cfg = O.make_config(O.BOUNCE, scheme, 0.01, hmax=0.05, events_on=True, evt_dir=(-1,),
                        evt_tol=(1e-12,))
    tr = O.trace_slice(cfg, [0.0, 12.0], [h0, 0.0], [g, r_])
    v = math.sqrt(2 * g * h0)
    t_exp, v_exp, tk = [], [], math.sqrt(2 * h0 / g)
    while tk < 12.0:
        t_exp.append(tk)
        v_exp.append(-v)
        tk += 2 * r_ * v / g
        v *= r_
    m = len(tr["ev_t"])
    assert m == len(t_exp) >= 5
    np.testing.assert_allclose(tr["ev_t"], t_exp, rtol=0, atol=1e-9)
    np.testing.assert_allclose(tr["ev_y"][:, 1], v_exp, rtol=1e-9)
    # velocity ratio between consecutive impacts is the restitution coefficient
    np.testing.assert_allclose(tr["ev_y"][1:, 1] / tr["ev_y"][:-1, 1], r_, rtol=1e-9)
    # every located point sits inside the event zone |y1| <= tol
    assert np.all(np.abs(tr["ev_y"][:, 0]) <= 1e-12)
    # event accessories keep the last impact (time, velocity before it)
    assert tr["acc"][4] == tr["ev_t"][-1] and tr["acc"][5] == tr["ev_y"][-1, 1]


# --------------------------------------------------------------------------
# Event location against a library integrator with its own root finder.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [0.2, 0.25, 0.3])
def test_duffing_event_times_against_scipy(k):
    from scipy.integrate import solve_ivp
    B, T = 0.3, 3 * 2 * math.pi
    f = lambda t, y: [y[1], -y[0] - y[0] ** 3 - k * y[1] + B * math.cos(t)]
    ev = lambda t, y: y[1]
    ev.direction = -1
    s = solve_ivp(f, (0, T), [-0.5, 0.1], method="DOP853", rtol=1e-13, atol=1e-14, events=ev)
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=1e-11, atol=1e-11, events_on=True,
                        evt_dir=(-1,), evt_tol=(1e-12,))
    tr = O.trace_slice(cfg, [0.0, T], [-0.5, 0.1], [k, B])
    assert len(tr["ev_t"]) == len(s.t_events[0]) >= 2
    np.testing.assert_allclose(tr["ev_t"], s.t_events[0], rtol=0, atol=1e-8)
    np.testing.assert_allclose(tr["ev_y"][:, 0], s.y_events[0][:, 0], rtol=0, atol=1e-9)


# --------------------------------------------------------------------------
# Lyapunov model, Eqs. (3)-(7): the polar linearisation (radius y3, angle y4)
# against the tangent flow written in Cartesian coordinates, u' = v,
# v' = g1 u + g2 v, with the radius reset at every slice end.
# --------------------------------------------------------------------------
def _lyap_oracle(mc, k, B, y0, n_per, rtol=1e-12):
    cfg = O.make_config(O.DUFFING_LYAPUNOV, O.RKCK45, 1e-2, rtol=rtol, atol=rtol, mc=mc,
                        td_mode=O.TD_SHIFT)
    N = len(k)
    td = np.vstack([np.zeros(N), np.full(N, 2 * math.pi)])
    r = O.run(cfg, td, np.asarray(y0, dtype=float), np.vstack([k, B]), n_slices=n_per, record=True)
    assert np.all(r["status"] == O.ST_TEND)
    return r["records"]  # (slice, A + n + 1, N), A = 5: a4 = ln y3 of the slice


def test_lyapunov_linear_oscillator_matches_matrix_exponential():
    # delta = -1, c3 = 0: constant tangent matrix J = [[0, 1], [-1, -k]], so
    # over slice s the tangent vector is expm(J T) applied s times to
    # (cos phi0, sin phi0); the slice's ln-stretch and end direction follow.
    from scipy.linalg import expm
    k = np.array([0.05, 0.2, 0.7, 1.3])
    phi0 = np.array([0.3, -1.0, 2.0, 4.0])
    N, n_per, T = len(k), 4, 2 * math.pi
    y0 = np.vstack([np.full(N, -0.5), np.full(N, 0.1), np.ones(N), phi0])
    rec = _lyap_oracle((-1.0, 0.0, 1.0), k, np.full(N, 0.3), y0, n_per)
    for i in range(N):
        M = expm(np.array([[0.0, 1.0], [-1.0, -k[i]]]) * T)
        e = np.array([math.cos(phi0[i]), math.sin(phi0[i])])
        for s_ in range(n_per):
            e_new = M @ e
            stretch = math.log(np.linalg.norm(e_new) / np.linalg.norm(e))
            e = e_new
            assert abs(rec[s_, 4, i] - stretch) < 1e-9
            assert rec[s_, 5 + 2, i] == 1.0  # radius reset to one
            d = e / np.linalg.norm(e)
            assert abs(rec[s_, 5 + 3, i]) <= math.pi  # angle reduced at the slice end
            assert abs(math.cos(rec[s_, 5 + 3, i]) - d[0]) < 1e-9
            assert abs(math.sin(rec[s_, 5 + 3, i]) - d[1]) < 1e-9


def test_lyapunov_linear_oscillator_exponent_is_minus_half_damping():
    # the largest exponent of x'' + k x' + x = B cos t is -k / 2 (k < 2); the
    # mean of ln y3 per unit time over n periods differs from it by a
    # bounded term / (n T)
    k = np.array([0.1, 0.4, 1.0])
    N, n_per, T = len(k), 200, 2 * math.pi
    y0 = np.vstack([np.full(N, -0.5), np.full(N, 0.1), np.ones(N), np.zeros(N)])
    rec = _lyap_oracle((-1.0, 0.0, 1.0), k, np.full(N, 0.3), y0, n_per, rtol=1e-10)
    lam = rec[:, 4, :].sum(axis=0) / (n_per * T)
    np.testing.assert_allclose(lam, -k / 2, rtol=0, atol=5e-4)


@pytest.mark.parametrize("delta", [-1.0, 1.0])
def test_lyapunov_nonlinear_against_cartesian_tangent_flow(delta):
    from scipy.integrate import solve_ivp
    k, B, n_per, T = 0.25, 0.3, 3, 2 * math.pi
    phi0 = 0.7

    def f(t, z):
        y1, y2, u, v = z
        g1 = delta - 3.0 * y1 * y1
        return [y2, delta * y1 - y1 ** 3 - k * y2 + B * math.cos(t), v, g1 * u - k * v]

    z0 = [-0.5, 0.1, math.cos(phi0), math.sin(phi0)]
    sol = solve_ivp(f, (0, n_per * T), z0, method="DOP853", rtol=1e-13, atol=1e-14,
                    t_eval=[T * (s_ + 1) for s_ in range(n_per)])
    rec = _lyap_oracle((delta, 1.0, 1.0), np.array([k]), np.array([B]),
                       np.array([[-0.5], [0.1], [1.0], [phi0]]), n_per)
    norm_prev = 1.0
    for s_ in range(n_per):
        y1, y2, u, v = sol.y[:, s_]
        nrm = math.hypot(u, v)
        # ln of the slice's stretch: the reset makes the stretches telescope
        assert abs(rec[s_, 4, 0] - math.log(nrm / norm_prev)) < 1e-8
        norm_prev = nrm
        assert abs(rec[s_, 5 + 0, 0] - y1) < 1e-9 and abs(rec[s_, 5 + 1, 0] - y2) < 1e-9
        assert abs(math.cos(rec[s_, 5 + 3, 0]) - u / nrm) < 1e-8
        assert abs(math.sin(rec[s_, 5 + 3, 0]) - v / nrm) < 1e-8


def test_event_brute_force_tiny():
    """Brute force: sample F on a fine fixed grid of an independent integration
    and bracket every downward crossing; each located time lies in a bracket."""
    from scipy.integrate import solve_ivp
    for k in (0.21, 0.27):
        B, T = 0.3, 2 * 2 * math.pi
        f = lambda t, y: [y[1], -y[0] - y[0] ** 3 - k * y[1] + B * math.cos(t)]
        grid = np.linspace(0, T, 200001)
        s = solve_ivp(f, (0, T), [-0.5, 0.1], method="DOP853", rtol=1e-13, atol=1e-14, t_eval=grid)
        F = s.y[1]
        brackets = [(grid[i], grid[i + 1]) for i in range(len(grid) - 1) if F[i] > 0 >= F[i + 1]]
        cfg = O.make_config(O.DUFFING, O.RK4, 1e-3, events_on=True, evt_dir=(-1,),
                            evt_tol=(1e-10,))
        tr = O.trace_slice(cfg, [0.0, T], [-0.5, 0.1], [k, B])
        assert len(tr["ev_t"]) == len(brackets)
        for te, (a, b) in zip(tr["ev_t"], brackets):
            assert a - 1e-6 <= te <= b + 1e-6


def test_event_inside_zone_at_start_is_not_detected():
    """A trajectory starting at a local maximum (y2 = 0) is in the leaving
    state; the first detection is the next maximum (Sec. 4, Sec. 7.2)."""
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(-1,), evt_tol=(1e-6,))
    # exactly at the maximum, and inside the zone just before it (y2 > 0)
    for y2 in (0.0, 5e-7):
        tr = O.trace_slice(cfg, [0.0, 4 * math.pi], [1.0, y2], [0.25, 0.3])
        assert len(tr["ev_t"]) >= 1
        assert tr["ev_t"][0] > 1.0


def test_wrong_direction_crossings_are_ignored():
    cfg_max = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(-1,), evt_tol=(1e-9,))
    cfg_min = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(1,), evt_tol=(1e-9,))
    cfg_any = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(0,), evt_tol=(1e-9,))
    args = ([0.0, 6 * math.pi], [-0.5, 0.1], [0.25, 0.3])
    a, b, c = (O.trace_slice(cfg, *args) for cfg in (cfg_max, cfg_min, cfg_any))
    # maxima have y1'' < 0, minima y1'' > 0
    for tr, sign in ((a, -1), (b, 1)):
        acc = [O.rhs(cfg_max, t, y, [0.25, 0.3])[1] for t, y in zip(tr["ev_t"], tr["ev_y"])]
        assert all(np.sign(x) == sign for x in acc)
    assert len(c["ev_t"]) == len(a["ev_t"]) + len(b["ev_t"])


# --------------------------------------------------------------------------
# Accessories (Sec. 5, Sec. 6.7): discrete max / min over accepted points.
# --------------------------------------------------------------------------
def test_accessories_equal_brute_force_over_accepted_points():
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(-1,), evt_tol=(1e-10,))
    tr = O.trace_slice(cfg, [0.0, 2 * math.pi], [-0.5, 0.1], [0.23, 0.3])
    y1 = tr["ys"][:, 0]
    i_max, i_min = int(np.argmax(y1)), int(np.argmin(y1))
    assert tr["acc"][0] == y1[i_max] and tr["acc"][1] == tr["t"][i_max]
    assert tr["acc"][2] == y1[i_min] and tr["acc"][3] == tr["t"][i_min]
    # event accessories: first detected maximum and the count
    assert tr["acc"][6] == len(tr["ev_t"])
    if len(tr["ev_t"]):
        assert tr["acc"][4] == tr["ev_y"][0, 0] and tr["acc"][5] == tr["ev_t"][0]


# --------------------------------------------------------------------------
# Step-size control (Sec. 6.5).
# --------------------------------------------------------------------------
def test_controller_step_counts_grow_as_tolerance_tightens():
    counts = []
    for tol in (1e-6, 1e-8, 1e-10, 1e-12):
        cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=tol, atol=tol)
        r = O.run(cfg, [[0.0], [2 * math.pi]], [[-0.5], [0.1]], [[0.25], [0.3]], n_slices=4)
        counts.append(int(r["nacc"][0]))
    assert counts == sorted(counts) and len(set(counts)) == 4
    # CK is fifth order: 100x tighter tolerance needs about 100^(1/5) = 2.5x steps
    for i in range(3):
        assert 1.8 < counts[i + 1] / counts[i] < 3.5


# Cash-Karp (1990) coefficients as published, in exact rationals, for the
# pins below (independent of the oracle's own tableau).
_CK_A = {(1, 0): Fraction(1, 5), (2, 0): Fraction(3, 40), (2, 1): Fraction(9, 40), (3, 0): Fraction(3, 10),
         (3, 1): Fraction(-9, 10), (3, 2): Fraction(6, 5), (4, 0): Fraction(-11, 54), (4, 1): Fraction(5, 2),
         (4, 2): Fraction(-70, 27), (4, 3): Fraction(35, 27), (5, 0): Fraction(1631, 55296),
         (5, 1): Fraction(175, 512), (5, 2): Fraction(575, 13824), (5, 3): Fraction(44275, 110592),
         (5, 4): Fraction(253, 4096)}
_CK_B5 = [Fraction(37, 378), 0, Fraction(250, 621), Fraction(125, 594), 0, Fraction(512, 1771)]
_CK_B4 = [Fraction(2825, 27648), 0, Fraction(18575, 48384), Fraction(13525, 55296), Fraction(277, 14336),
          Fraction(1, 4)]


def _ck_error_polynomial():
    """Coefficients P_k (k = 1..6) of the embedded error estimate on y' = lam y:
    e = P(z) y_n with z = lam h and P_k = (b5 - b4)^T A^(k-1) 1."""
    e = [Fraction(x) - Fraction(y) for x, y in zip(_CK_B5, _CK_B4)]
    v = [Fraction(1)] * 6
    coef = []
    for _ in range(6):
        coef.append(sum(e[i] * v[i] for i in range(6)))
        v = [sum(_CK_A.get((i, j), Fraction(0)) * v[j] for j in range(6)) for i in range(6)]
    return coef


def _controller_next(h, err, shrink=0.1, grow=5.0, hmin=1e-12, hmax=1e6):
    """The next step from the controller law of Sec. 3 / 6.5 (reading: factor
    0.9 err^(-1/5), clamped to [shrink, grow], step clamped to [hmin, hmax];
    err = 0 gives the grow limit)."""
    fac = grow if err == 0.0 else min(max(0.9 * math.pow(err, -0.2), shrink), grow)
    return min(max(h * fac, hmin), hmax)


def test_controller_next_step_recomputed_from_each_trial():
    """Every trial step's next step size (accepted and rejected ones) equals
    the controller law applied to that trial's own error vector, with the
    error ratio max_m |e_m| / (atol + rtol max(|y_n,m|, |y_n+1,m|))."""
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1.0, rtol=1e-9, atol=1e-9, mc=(-1.0, 0.0, 1.0))
    r = O.trace_slice(cfg, [0.0, 30.0], [1.0, 0.0], [0.05, 0.0], trial_cap=100000)
    T = r["trials"]
    assert (T["ok"] == 0).sum() >= 1 and (T["ok"] == 1).sum() > 100  # h0 = 1 is rejected first
    for k in range(len(T["h"])):
        sc = 1e-9 + 1e-9 * np.maximum(np.abs(T["y"][k]), np.abs(T["ynew"][k]))
        err = max(abs(T["e"][k][m]) / sc[m] for m in range(2))
        assert (err > 1.0) == (T["ok"][k] == 0)
        assert _controller_next(T["h"][k], err) == T["hnext"][k], k


def test_controller_settles_at_its_fixed_point():
    """On y2' = -y2 (Duffing with delta = c3 = B = 0, k = 1) the embedded error
    is P(-h) y2 with P fixed by the published tableau, so with a pure relative
    tolerance the error ratio depends on h alone and the controller
    h <- 0.9 err^(-1/5) h settles where err = 0.9^5.  The steady step of the
    oracle must equal that root (a safety factor of 0.8 moves it by 11 %, an
    exponent of -1/4 by 2 %)."""
    from scipy.optimize import brentq
    coef = _ck_error_polynomial()
    assert coef[:4] == [0, 0, 0, 0] and coef[4] != 0  # fourth-order embedded estimate
    rtol = 1e-10
    P = lambda z: sum(float(coef[k]) * z ** (k + 1) for k in range(6))
    hstar = brentq(lambda h: abs(P(-h)) / rtol - 0.9 ** 5, 1e-4, 2.0)
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, rtol=rtol, atol=1e-30, mc=(0.0, 0.0, 1.0))
    r = O.trace_slice(cfg, [0.0, 30.0], [0.0, 1.0], [1.0, 0.0], trial_cap=100000)
    T = r["trials"]
    sel = (T["ok"] == 1) & (T["t"] > 5.0) & (T["t"] < 25.0)
    assert sel.sum() > 300
    np.testing.assert_allclose(T["h"][sel], hstar, rtol=1e-7)


def test_nan_rejects_and_stops_at_hmin():
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, hmin=1e-6)
    r = O.run(cfg, [[0.0], [1.0]], [[-0.5], [0.1]], [[float("nan")], [0.3]])
    assert r["status"][0] == O.ST_HMIN_NAN
    # 1e-2 .. 1e-6 in factors of 10 (one more if rounding leaves h just above hmin)
    assert r["nacc"][0] == 0 and r["nrej"][0] in (5, 6)
    assert np.all(r["y"][:, 0] == [-0.5, 0.1])


def test_valve_negative_pressure_is_rejected_not_propagated():
    """sqrt of a negative chamber pressure gives NaN; the step is rejected and
    the controller retreats instead of stopping (Sec. 6.5)."""
    cfg = O.make_config(O.VALVE, O.RKCK45, 1.0, rtol=1e-9, atol=1e-9)
    r = O.run(cfg, [[0.0], [1.0]], [[0.5], [0.0], [1e-3]], [[1.25], [10.0], [20.0], [0.5], [0.8]])
    assert r["nrej"][0] >= 1
    assert r["status"][0] == O.ST_TEND and np.all(np.isfinite(r["y"][:, 0]))


def test_accept_at_minimum_step_without_tolerance():
    cfg = O.make_config(O.DUFFING, O.RKCK45, 0.5, rtol=1e-15, atol=1e-15, hmin=0.5, hmax=0.5)
    r = O.run(cfg, [[0.0], [5.0]], [[-0.5], [0.1]], [[0.25], [0.3]])
    assert r["nrej"][0] == 0 and r["nacc"][0] == 10 and r["status"][0] == O.ST_TEND


def test_step_budget_stops():
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-3, max_steps=10)
    r = O.run(cfg, [[0.0], [100.0]], [[-0.5], [0.1]], [[0.25], [0.3]])
    assert r["status"][0] == O.ST_STEP_BUDGET and r["nacc"][0] + r["nrej"][0] == 10


def test_rk4_fixed_grid_step_count():
    N = 3
    cfg = O.make_config(O.DUFFING, O.RK4, 2 * math.pi / 1000)
    r = O.run(cfg, [np.zeros(N), np.full(N, 2 * math.pi)], np.tile([[-0.5], [0.1]], N),
              np.vstack([np.linspace(0.2, 0.3, N), np.full(N, 0.3)]), n_slices=7)
    assert np.all(r["nacc"] == 7000) and np.all(r["nrej"] == 0)


# --------------------------------------------------------------------------
# Slices, finalization and records (Sec. 6.8, Sec. 7.1.1).
# --------------------------------------------------------------------------
def test_records_match_consecutive_single_slices():
    N = 3
    k = np.linspace(0.2, 0.3, N)
    p = np.vstack([k, np.full(N, 0.3)])
    td = [np.zeros(N), np.full(N, 2 * math.pi)]
    y = np.tile([[-0.5], [0.1]], N)
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(-1,), evt_tol=(1e-12,))
    whole = O.run(cfg, td, y, p, n_slices=4, n_skip=1, record=True)
    cur = dict(td=np.array(td), y=y, acc=None)
    for s in range(4):
        step = O.run(cfg, cur["td"], cur["y"], p, cur["acc"])
        if s >= 1:
            rec = whole["records"][s - 1]
            np.testing.assert_array_equal(rec[:7], step["acc"])
            np.testing.assert_array_equal(rec[7:9], step["y"])
            np.testing.assert_array_equal(rec[9], 2 * math.pi)
        cur = dict(td=step["td"], y=step["y"], acc=step["acc"])
    np.testing.assert_array_equal(whole["y"], cur["y"])


@pytest.mark.parametrize("mode", [O.TD_KEEP, O.TD_T0_TO_T, O.TD_SHIFT])
def test_time_domain_modes(mode):
    cfg = O.make_config(O.DUFFING, O.RKCK45, 1e-2, events_on=True, evt_dir=(-1,), evt_tol=(1e-8,),
                        evt_stop=(1,), td_mode=mode)
    r = O.run(cfg, [[0.0], [100.0]], [[-0.5], [0.1]], [[0.25], [0.3]], n_slices=3, record=True)
    t_end = r["records"][:, 9, 0]
    assert np.all(r["records"][:, 8, 0] <= 1e-8)  # every slice stopped at a maximum
    if mode == O.TD_KEEP:
        assert r["td"][0, 0] == 0.0 and r["td"][1, 0] == 100.0
        # every slice restarts at t0 = 0: the stop times are then equal only if
        # the state is periodic; they are at least all inside the domain
        assert np.all((t_end > 0) & (t_end < 100))
    elif mode == O.TD_T0_TO_T:
        assert r["td"][0, 0] == t_end[-1] and r["td"][1, 0] == 100.0
        assert np.all(np.diff(t_end) > 0)
    else:
        assert r["td"][0, 0] == t_end[-1]
        assert math.isclose(r["td"][1, 0] - r["td"][0, 0], 100.0 - 0.0 if False else r["td"][1, 0] - t_end[-1])
        assert np.all(np.diff(t_end) > 0)
    assert np.all(r["status"] == O.ST_EVENT_STOP)


# --------------------------------------------------------------------------
# Keller-Miksis (Sec. 2.2).
# --------------------------------------------------------------------------
def test_km_zero_amplitude_rests_at_equilibrium():
    """With P_A = 0, y = (1, 0) is an equilibrium because C0 - C2 - C3 = 0
    (Eqs. (16), (18), (19))."""
    C = O.km_coefficients([0.0], [2 * math.pi * 1e5])
    assert abs(C[0, 0] - C[2, 0] - C[3, 0]) <= 1e-12 * C[0, 0]
    # hmax keeps h inside the stability region: at rest the error estimate
    # vanishes and would otherwise let h grow far past the bubble period
    cfg = O.make_config(O.KELLER_MIKSIS, O.RKCK45, 1e-2, rtol=1e-10, atol=1e-10, hmax=0.01)
    r = O.run(cfg, [[0.0], [1.0]], [[1.0], [0.0]], C, n_slices=5)
    assert abs(r["y"][0, 0] - 1.0) < 1e-12 and abs(r["y"][1, 0]) < 1e-12
    # a perturbed bubble is driven back towards it by a restoring force
    f_plus = O.rhs(cfg, 0.0, [1.01, 0.0], C[:, 0])[1]
    f_minus = O.rhs(cfg, 0.0, [0.99, 0.0], C[:, 0])[1]
    assert f_plus < 0 < f_minus


def _km_dimensional(PA, f, T_periods, PA2=0.0, f2=None):
    """Independent integration of the dimensional Keller-Miksis equation,
    Eqs. (8)-(11), for R(t) in SI units (scipy DOP853), with one or two
    excitation frequencies (theta = 0)."""
    from scipy.integrate import solve_ivp
    ph = O.KM_WATER
    rho, c, sig, mu, pV, Pinf, gam, RE = (ph[k] for k in ("rho", "cL", "sigma", "mu", "pV", "Pinf",
                                                          "gamma", "RE"))
    w = 2 * math.pi * f
    w2 = 2 * math.pi * (f if f2 is None else f2)
    Pg0 = Pinf - pV + 2 * sig / RE

    def rhs(t, u):
        R, Rd = u
        pG = Pg0 * (RE / R) ** (3 * gam)
        pL = pG + pV - 2 * sig / R - 4 * mu * Rd / R
        pinf = Pinf + PA * math.sin(w * t) + PA2 * math.sin(w2 * t)
        # d/dt (p_L - p_inf) without its R'' part, which is moved to the left
        dp = (-3 * gam * pG * Rd / R + 2 * sig * Rd / R ** 2 + 4 * mu * Rd ** 2 / R ** 2
              - PA * w * math.cos(w * t) - PA2 * w2 * math.cos(w2 * t))
        lhs = (1 - Rd / c) * R + 4 * mu / (rho * c)
        rhs_ = (1 + Rd / c) * (pL - pinf) / rho + R / (rho * c) * dp - (1 - Rd / (3 * c)) * 1.5 * Rd ** 2
        return [Rd, rhs_ / lhs]

    s = solve_ivp(rhs, (0, T_periods / f), [RE, 0.0], method="DOP853", rtol=1e-12, atol=1e-20,
                  t_eval=np.arange(1, T_periods + 1) / f)
    return s.y[0] / RE, s.y[1] / RE / f


@pytest.mark.parametrize("PA,f", [(0.5e5, 100e3), (1.2e5, 300e3)])
def test_km_dimensionless_matches_dimensional(PA, f):
    C = O.km_coefficients([PA], [2 * math.pi * f])
    cfg = O.make_config(O.KELLER_MIKSIS, O.RKCK45, 1e-3, rtol=1e-12, atol=1e-12)
    r = O.run(cfg, [[0.0], [1.0]], [[1.0], [0.0]], C, n_slices=3, record=True)
    y1_ref, y2_ref = _km_dimensional(PA, f, 3)
    np.testing.assert_allclose(r["records"][:, 4, 0], y1_ref, rtol=1e-8)
    np.testing.assert_allclose(r["records"][:, 5, 0], y2_ref, rtol=1e-6, atol=1e-8)


def test_km_dual_frequency_matches_dimensional():
    """Two excitation frequencies (Eq. (9)): the dimensionless Eqs. (12)-(28)
    against the dimensional Eqs. (8)-(11).  This pins C8 to omega_2 (the
    printed omega_1 is off by 0.4 % here)."""
    PA1, PA2, f1, f2 = 0.5e5, 0.7e5, 100e3, 170e3
    C = O.km_coefficients([PA1], [2 * math.pi * f1], PA2=PA2, omega2=2 * math.pi * f2, theta=0.0)
    assert C[11, 0] == f2 / f1
    cfg = O.make_config(O.KELLER_MIKSIS, O.RKCK45, 1e-3, rtol=1e-12, atol=1e-12, td_mode=O.TD_SHIFT)
    r = O.run(cfg, [[0.0], [1.0]], [[1.0], [0.0]], C, n_slices=3, record=True)
    y1_ref, _ = _km_dimensional(PA1, f1, 3, PA2=PA2, f2=f2)
    np.testing.assert_allclose(r["records"][:, 4, 0], y1_ref, rtol=1e-8)


# --------------------------------------------------------------------------
# Pressure relief valve (Sec. 2.3, Sec. 7.3).
# --------------------------------------------------------------------------
def _valve_cfg(**kw):
    ev = GOLD["event_properties"]
    return O.make_config(O.VALVE, O.RKCK45, 1e-2, rtol=1e-10, atol=1e-10, events_on=True,
                         evt_dir=ev["direction"], evt_tol=ev["tolerance"], evt_stop=ev["stop"],
                         max_eq=ev["max_iteration_for_equilibrium"], td_mode=O.TD_SHIFT, **kw)


def _valve_params(q):
    v = GOLD["valve"]
    return [[v["kappa"]], [v["delta"]], [v["beta"]], [q], [v["r"]]]


def _valve_two_event_trace(direction, y0, delta, T=3.0):
    """One valve slice with both events on and a fixed step h = 1 long enough
    to cross both event surfaces in one step (kappa 1.25, beta 0.1, q 1,
    r 0.8; event tolerances 1e-10).  Also returns the end of that first step
    without location, to show both surfaces were crossed in it."""
    p = [1.25, delta, 0.1, 1.0, 0.8]
    cfg = O.make_config(O.VALVE, O.RKCK45, 1.0, rtol=1e-6, atol=1e-6, hmin=1.0, hmax=1.0, events_on=True,
                        evt_dir=direction, evt_tol=(1e-10, 1e-10), evt_stop=(0, 0), max_eq=0)
    y1, _ = O.single_step(cfg, 0.0, y0, p, 1.0)
    return O.trace_slice(cfg, [0.0, T], y0, p), p, y1


def _valve_free_flight(p, y0, T):
    """Independent integration of Eqs. (29)-(31) without events (scipy)."""
    from scipy.integrate import solve_ivp
    kap, dl, bt, q, _ = p
    f = lambda t, y: [y[1], -kap * y[1] - (y[0] + dl) + y[2], bt * (q - y[0] * math.sqrt(max(y[2], 0.0)))]
    grid = np.linspace(0.0, T, 300001)
    return grid, solve_ivp(f, (0.0, T), y0, method="DOP853", rtol=1e-12, atol=1e-13, t_eval=grid).y


def test_second_event_fires_at_the_located_point_only_if_crossed_there():
    """Sec. 4: when several events are detected in one step only the highest
    index is located.  Here one step of size 1 first crosses the impact
    surface y1 = 0 (event 1, downwards) and only later (on the un-impacted
    flow) the minimum y2 = 0 (event 0, upwards).  At the located impact y2 is
    still negative, so event 0 must not fire there; brute force on an
    independent integration confirms that y2 < 0 all the way to the impact."""
    y0 = [0.01, -1.0, 1.0]
    r, p, yend = _valve_two_event_trace((+1, -1), y0, delta=0.5)
    assert yend[0] < 0.0 and yend[1] > 0.0  # the whole step crossed both surfaces
    grid, Y = _valve_free_flight(p, y0, 1.0)
    i = int(np.argmax(Y[0] <= 0.0))  # first grid point past the impact
    assert i > 0 and np.all(Y[1][: i + 1] < 0.0)
    # the one-step location is within the step's own accuracy of the impact
    assert r["ev_index"][0] == 1 and abs(r["ev_t"][0] - grid[i]) < 1e-3
    # ... and the minimum of the flow without the impact comes later in that step
    assert np.any(Y[1][i:] > 0.0)
    assert 0 not in list(r["ev_index"][r["ev_t"] <= r["ev_t"][0]])


def test_second_event_crossed_before_the_located_point_fires_with_it():
    """The other case of the same rule: the step first passes a maximum
    (event 0, y2 falling through 0) and then the impact (event 1).  Event 1 is
    located; event 0 is still crossed at that point and fires there, in
    ascending order, before the impact action."""
    y0 = [0.05, 0.1, 1.0]
    r, p, yend = _valve_two_event_trace((-1, -1), y0, delta=2.0)
    assert yend[0] < 0.0 and yend[1] < 0.0  # the whole step crossed both surfaces
    grid, Y = _valve_free_flight(p, y0, 1.0)
    i_max = int(np.argmax(Y[1] <= 0.0))
    i_imp = int(np.argmax(Y[0] <= 0.0))
    assert 0 < i_max < i_imp  # maximum first, impact later, both within the first step
    assert list(r["ev_index"][:2]) == [0, 1]
    assert r["ev_t"][0] == r["ev_t"][1] and abs(r["ev_t"][1] - grid[i_imp]) < 1e-3
    # event 0 saw the pre-action state (y2 < 0), the impact then reversed y2
    assert r["ev_y"][0][1] < 0 and r["ev_y_after"][1][1] == -0.8 * r["ev_y"][1][1]


def test_valve_high_flow_rate_settles_to_equilibrium():
    from scipy.optimize import brentq
    q, delta = 9.5, GOLD["valve"]["delta"]
    r = O.run(_valve_cfg(), [[0.0], [1e3]], [[0.2], [0.0], [delta]], _valve_params(q), n_slices=300,
              record=True)
    assert r["status"][0] == O.ST_EQUILIBRIUM
    y1s = brentq(lambda x: x * math.sqrt(x + delta) - q, 0.0, 10.0)
    y1, y2, y3 = r["y"][:, 0]
    assert abs(y2) <= 1e-6
    assert abs(y1 - y1s) < 1e-3 and abs(y3 - (y1s + delta)) < 1e-2
    # max and min of the last slice coincide at equilibrium (Sec. 7.3)
    assert abs(r["acc"][0, 0] - r["acc"][2, 0]) < 1e-3


def test_valve_impact_law():
    """Eqs. (32)-(34) at every located impact: y1 stays at the seat (within
    the event tolerance), y2+ = -r y2-, y3 is continuous."""
    r_coef = GOLD["valve"]["r"]
    cfg = _valve_cfg()
    p = np.array(_valve_params(2.0))
    first = O.run(cfg, [[0.0], [1e3]], [[0.2], [0.0], [10.0]], p)  # up to the first maximum
    tr = O.trace_slice(cfg, first["td"][:, 0], first["y"][:, 0], p[:, 0])  # falls onto the seat
    imp = tr["ev_index"] == 1
    assert imp.sum() >= 1
    before, after = tr["ev_y"][imp], tr["ev_y_after"][imp]
    assert np.all(before[:, 1] < 0)
    np.testing.assert_array_equal(after[:, 1], -r_coef * before[:, 1])
    np.testing.assert_array_equal(after[:, 0], before[:, 0])
    np.testing.assert_array_equal(after[:, 2], before[:, 2])
    assert np.all(np.abs(before[:, 0]) <= cfg.evt_tol[1])


def test_valve_low_flow_rate_impacts():
    r = O.run(_valve_cfg(), [[0.0], [1e3]], [[0.2], [0.0], [10.0]], _valve_params(2.0), n_slices=40,
              n_skip=20, record=True)
    rec = r["records"]
    assert np.all(r["status"] == O.ST_EVENT_STOP)
    # every recorded iteration runs max -> max and touches the seat
    assert np.all(rec[:, 4, 0] >= 1)  # impacts per iteration
    assert np.all(np.abs(rec[:, 2, 0]) <= 1e-6)  # min y1 at the seat (inside the zone)
    assert np.all(rec[:, 0, 0] > 0.1)
