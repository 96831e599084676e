"""Pins of the oracle's 0D models (Section 2.1.2) and the smoothing of Section 2.2.1."""
import math

import numpy as np
import pytest

import golden_fixtures
import oracle
from workloads import profiles

# ---- S(t, t0, L_S), Eq. SmoothFunction ------------------------------------


def test_smooth_limits_and_monotone():
    ex = golden_fixtures.load("smoothing_example_section2_2_1.txt")  # T_d = 0.5 s, N_S = 15, dt = 0.005 s
    t0, dt, ns = ex["t0_s"], ex["dt_s"], ex["N_S"]
    LS = ns * dt
    assert oracle.smooth(t0 - 1e-9, t0, LS) == 1.0
    assert oracle.smooth(0.0, t0, LS) == 1.0
    assert oracle.smooth(t0, t0, LS) == 1.0
    assert oracle.smooth(t0 + LS, t0, LS) == 0.0
    assert oracle.smooth(t0 + LS + 1e-9, t0, LS) == 0.0
    ts = t0 + LS * np.linspace(0.0, 1.0, 2001)
    s = np.array([oracle.smooth(t, t0, LS) for t in ts])
    assert np.all((s >= 0) & (s <= 1)) and np.all(np.diff(s) <= 0)   # monotone in [0, 1]
    inner = (ts > t0 + 0.1 * LS) & (ts < t0 + 0.9 * LS)
    assert np.all((s[inner] > 0) & (s[inner] < 1))
    assert np.all(np.diff(s[inner]) < 0)   # strictly decreasing away from the flat ends
    # the 15 steps of the example stay strictly inside (0, 1] and reach 0 at the end
    steps = [oracle.smooth(t0 + k * dt, t0, LS) for k in range(ns + 1)]
    assert steps[0] == 1.0 and steps[-1] == 0.0 and all(0 < x < 1 for x in steps[1:-1])


def test_smooth_midpoint_value_and_flat_ends():
    # at u = 1/2 the definition gives exp(2 e^{-2} / (-1/2)) = exp(-4/e^2)
    assert oracle.smooth(1.5, 1.0, 1.0) == pytest.approx(math.exp(-4.0 / math.e ** 2), rel=1e-15)
    ex = golden_fixtures.load("smoothing_example_section2_2_1.txt")
    t0, LS = ex["t0_s"], ex["N_S"] * ex["dt_s"]
    assert oracle.smooth(t0 + 0.5 * LS, t0, LS) == pytest.approx(math.exp(-4.0 / math.e ** 2), rel=1e-14)
    # C-infinity: one-sided slopes vanish at both ends of the window
    h = 1e-4
    d0 = (oracle.smooth(h, 0.0, 1.0) - 1.0) / h
    d1 = (oracle.smooth(1.0, 0.0, 1.0) - oracle.smooth(1.0 - h, 0.0, 1.0)) / h
    assert abs(d0) < 1e-12 and abs(d1) < 1e-12


# ---- three-element Windkessel, Eqs. rightbc / rightQ ----------------------

RP, C, RD = 0.05, 200.0, 1.0


def test_rcr_free_decay_closed_form():
    # Q = 0: the discrete recursion is P_w,n = P_w,0 (1 - dt/(R_d C))^n exactly
    Pw = 0.01
    for n in range(1, 2001):
        Pw, P = oracle.rcr_step(Pw, 0.0, RP, C, RD)
        if n in (1, 10, 500, 2000):
            assert Pw == pytest.approx(0.01 * (1 - 1 / (RD * C)) ** n, rel=1e-12)
            assert P == Pw                       # no flow, no drop across Z_w
    # and it tends to the continuous RC decay e^{-t/(R_d C)} as dt -> 0 (first order)
    assert 0.01 * (1 - 1 / (RD * C)) ** 2000 == pytest.approx(0.01 * math.exp(-2000 / (RD * C)), rel=0.06)


def test_rcr_matches_paper_form():
    # one step from (P_w, Q): the increment equals Eq. rightbc evaluated with the
    # boundary pressure of Eq. rightQ, P = P_w + Z_w Q  (Z_w = R_p, C_w = C, R_w = R_d)
    rng = np.random.default_rng(3)
    for _ in range(20):
        Pw0, Q = rng.uniform(-0.01, 0.01), rng.uniform(-0.02, 0.02)
        Pw1, P1 = oracle.rcr_step(Pw0, Q, RP, C, RD)
        Pb = Pw0 + RP * Q
        rhs = Pb / (C * RP) - (RD + RP) / (C * RD * RP) * Pw0
        assert Pw1 - Pw0 == pytest.approx(rhs, rel=1e-9, abs=1e-18)
        assert (P1 - Pw1) / RP == pytest.approx(Q, rel=1e-12)        # Eq. rightQ at t_{n+1}


def test_rcr_steady_and_sinusoidal_response():
    # constant outflow q: P_w -> R_d q, P -> (R_d + R_p) q
    Pw, q = 0.0, 0.01
    for _ in range(20000):
        Pw, P = oracle.rcr_step(Pw, q, RP, C, RD)
    assert Pw == pytest.approx(RD * q, rel=1e-12) and P == pytest.approx((RD + RP) * q, rel=1e-12)
    # sinusoidal q_n = q0 cos(w n): steady discrete response P_w,n = Re{A e^{i w n}},
    # A (e^{i w} - a) = q0 / C with a = 1 - 1/(R_d C)   (z-transform of the recursion)
    w, q0 = 2 * math.pi / 1000, 0.01
    a = 1 - 1 / (RD * C)
    A = (q0 / C) / (np.exp(1j * w) - a)
    Pw, n_end = 0.0, 40000
    for n in range(n_end):
        Pw, P = oracle.rcr_step(Pw, q0 * math.cos(w * n), RP, C, RD)
    assert Pw == pytest.approx((A * np.exp(1j * w * n_end)).real, abs=1e-14)
    # continuous transfer |H| = (1/C)/sqrt(w^2 + (1/(R_d C))^2) to O(dt)
    assert abs(A) == pytest.approx(q0 / C / math.sqrt(w ** 2 + (1 / (RD * C)) ** 2), rel=2e-2)


# ---- LV elastance ODE, Eq. LVE -------------------------------------------


def test_lv_ode_constant_elastance_exact():
    # E' = 0: dP_v/dt = -E Q, forward Euler is exact for constant Q
    Pv = 0.003
    for _ in range(100):
        Pv = oracle.lv_ode(Pv, 2e-3, 0.0, 0.01)
    assert Pv == pytest.approx(0.003 - 100 * 2e-3 * 0.01, rel=1e-12)


def test_lv_volume_invariant_first_order():
    # with Q = 0 the continuous ODE keeps C_v P_v = P_v / E constant; forward Euler
    # keeps it to O(dt): halving dt (doubling the steps per beat) halves the drift
    drifts = []
    for T in (500, 1000, 2000, 4000):
        tab = profiles.elastance_table(T, 1e-3, 3e-5)
        Pv = 1e-3
        v0 = Pv / tab[0, 0]
        for n in range(int(0.3 * T)):                  # through the contraction
            Pv = oracle.lv_ode(Pv, tab[n, 0], tab[n, 1], 0.0)
        drifts.append(abs(Pv / tab[int(0.3 * T), 0] - v0) / v0)
    ratios = [drifts[i] / drifts[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (drifts, ratios)


def test_elastance_table_inputs():
    T = 4000
    tab = profiles.elastance_table(T, 2.0, 0.06)
    assert tab[:, 0].max() == pytest.approx(2.0, rel=1e-6)
    assert tab[:, 0].min() == pytest.approx(0.06, rel=1e-3)
    # analytic derivative agrees with central differences of the same curve
    fd = (np.roll(tab[:, 0], -1) - np.roll(tab[:, 0], 1)) / 2.0
    sl = slice(5, T - 5)
    assert np.allclose(tab[sl, 1], fd[sl], atol=2e-3 * np.abs(fd).max())


def test_lv_valve_logic():
    # opens when P_v exceeds the inlet gauge pressure, not tested for closure on that step
    Pv, op, Td, closed = oracle.lv_step(0.001, 0.0, -1e300, 10, 1e-3, 1e-5, -0.5, 0.0, 1e-3)
    assert op == 1.0 and closed == 0
    # closes at the first step with Q < 0, recording T_d = t_n
    Pv, op, Td, closed = oracle.lv_step(Pv, op, Td, 11, 1e-3, 0.0, -1e-4, 0.0, 1e-3)
    assert op == 0.0 and Td == 11.0 and closed == 1
    # while closed P_v never drops below the atrial pressure (ideal mitral diode)
    Pv, op, Td, closed = oracle.lv_step(0.0002, 0.0, 11.0, 12, 1e-3, -1e-4, 0.0, 0.01, 1e-3)
    assert Pv == 1e-3 and op == 0.0


def _closed_loop(T, beats=12):
    kappa = 4.9e-4
    tab = profiles.elastance_table(T, 2.0 * kappa, 0.06 * kappa)
    # resistances scale with the steps per beat so that only dt changes with T
    Rp, Cw, Rd, P_la = 0.05 * T / 2000, 200.0, 1.0 * T / 2000, 1e-3
    Pv, op, Td, Pw, Q = P_la, 0.0, -1e300, 0.0, 0.0
    out = []
    for beat in range(beats):
        flow, opens, v_open, v_close = 0.0, 0, None, None
        for m in range(T):
            n = beat * T + m
            E, Ed = tab[n % T]
            Pin = Pv if op else Pw + Rp * Q
            was = op
            Pv, op, Td, _ = oracle.lv_step(Pv, op, Td, n, E, Ed, Q, Pin, P_la)
            vol = Pv / tab[(n + 1) % T, 0]
            if op == 1.0 and was == 0.0:
                opens += 1
                v_open = vol
            if op == 0.0 and was == 1.0:
                v_close = vol
            Q = (Pv - Pw) / Rp if op else 0.0
            Pw, _ = oracle.rcr_step(Pw, Q, Rp, Cw, Rd)
            flow += Q
        out.append((flow, opens, v_open, v_close))
    return out


def test_closed_loop_pv_loop_periodic():
    """0D-only loop: the LV ejects through Z_w = R_p into the Windkessel chamber,
    Q = (P_v - P_w)/R_p while the valve is open.  The loop becomes periodic with
    one opening per beat, and the ventricular volume lost during ejection equals
    the ejected volume (V' = -Q) up to the first-order error of forward Euler,
    which halves when the beat is resolved with twice the steps."""
    errs = []
    for T in (1000, 2000, 4000):
        res = _closed_loop(T)
        (fl1, o1, _, _), (fl2, o2, vo, vc) = res[-2], res[-1]
        assert o1 == 1 and o2 == 1
        assert abs(fl2 - fl1) / fl2 < 1e-6
        errs.append(abs((vo - vc) - fl2) / fl2)
    assert errs[0] < 0.12
    assert 1.8 < errs[0] / errs[1] < 2.3 and 1.8 < errs[1] / errs[2] < 2.3, errs


# ---- higher-order marching (Heun RK2, classical RK4) ----------------------

@pytest.mark.parametrize("order", [2, 4])
def test_rcr_higher_order_stability_polynomial(order):
    # Q = 0: one step multiplies P_w by the method's stability polynomial
    # R(z) at z = -dt/(R_d C): 1 + z + z^2/2 (RK2), + z^3/6 + z^4/24 (RK4)
    z = -1.0 / (RD * C)
    R = 1 + z + z * z / 2 + ((z ** 3 / 6 + z ** 4 / 24) if order == 4 else 0.0)
    Pw = 0.01
    for n in range(1, 301):
        Pw, P = oracle.rcr_step_ord(Pw, 0.0, RP, C, RD, order)
    assert Pw == pytest.approx(0.01 * R ** 300, rel=1e-12)


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 4.0), (4, 16.0)])
def test_rcr_convergence_order(order, ratio):
    # sinusoidal outflow over one period of fixed length, resolved with M
    # steps (C scaled with M so the time constant stays 0.2 of the period);
    # error against the exact solution of the linear ODE with the input held
    # piecewise constant, e^{-h/tau}-recursion, shrinks by 2^order per halving
    errs = []
    for M in (200, 400, 800):
        Cm = 200.0 * M / 1000.0
        Pw_num = Pw_ex = 0.0
        a = math.exp(-1.0 / (RD * Cm))
        for n in range(M):
            q = 0.01 * math.cos(2 * math.pi * n / M)
            Pw_num, _ = oracle.rcr_step_ord(Pw_num, q, RP, Cm, RD, order)
            Pw_ex = a * Pw_ex + RD * q * (1 - a)     # exact over a step with q held
        errs.append(abs(Pw_num - Pw_ex))
    r = errs[0] / errs[1], errs[1] / errs[2]
    assert all(0.8 * ratio < x < 1.25 * ratio for x in r), (errs, r)


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 4.0), (4, 16.0)])
def test_lv_invariant_higher_order(order, ratio):
    # Q = 0 keeps C_v P_v = P_v / E constant; with a smooth elastance
    # E(t) = a (1 + sin(2 pi t / T) / 2) the drift over 0.3 of a beat falls by
    # 2^order per halving of dt (the double-Hill curve is not smooth at the
    # beat start, t^1.32, so it would cap the observed order)
    drifts = []
    for T in (100, 200, 400):
        n = np.arange(T + 1)
        E = 1e-3 * (1 + 0.5 * np.sin(2 * np.pi * n / T))
        D = 1e-3 * 0.5 * (2 * np.pi / T) * np.cos(2 * np.pi * n / T)
        Pv = 1e-3
        v0 = Pv / E[0]
        m = int(round(0.3 * T))
        for k in range(m):
            Pv = oracle.lv_ode_ord(Pv, E[k], D[k], E[k + 1], D[k + 1], 0.0, order)
        drifts.append(abs(Pv / E[m] - v0) / v0)
    r = drifts[0] / drifts[1], drifts[1] / drifts[2]
    assert all(0.8 * ratio < x < 1.25 * ratio for x in r), (drifts, r)


def test_lv_higher_order_exact_for_constant_elastance():
    for order in (2, 4):
        Pv = 0.003
        for _ in range(100):
            Pv = oracle.lv_ode_ord(Pv, 2e-3, 0.0, 2e-3, 0.0, 0.01, order)
        assert Pv == pytest.approx(0.003 - 100 * 2e-3 * 0.01, rel=1e-12)
