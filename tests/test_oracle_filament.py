"""Pins of the oracle's SGFD filament solid (Section 2.3.2, Eqs. tension,
2nd order, bending) and of its coupling into the wall-node update.

* closed forms of the difference operators: a rigid motion and an
  unstretched straight line carry no force; the tension operator is exact on
  a quadratic stretch, the bending operator on a quartic (force -24 EI);
* the method of manufactured solutions of Section 3.1 (Eq. MMSsolid): the
  error of the marched filament against X = (s, A cos(pi s) sin(pi t)) falls
  as ds^2;
* a pre-tensioned, simply supported filament on the lattice (penalty off)
  oscillates in its sine mode exactly as the discrete dispersion relation of
  the central-difference scheme predicts.
"""
import numpy as np
import pytest

import golden_fixtures
import oracle
from workloads import IBNodes, Instance, geometry


def _ghosts_from(fun, s, ds):
    return fun(np.array([s[0] - ds]))[0], fun(np.array([s[-1] + ds]))[0]


def test_rigid_motion_and_unstretched_line_carry_no_force():
    rng = np.random.default_rng(0)
    n, ds = 12, 0.7
    s = np.arange(n) * ds
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    line = lambda ss: np.stack([ss, 0 * ss, 0 * ss], axis=1) @ R.T + np.array([1.0, -2.0, 0.5])
    gl, gr = _ghosts_from(line, s, ds)
    F = oracle.filament_force(line(s), gl, gr, ds, 3.0, 0.2)
    assert np.abs(F).max() < 1e-12
    assert np.all(F[[0, -1]] == 0.0)


def test_tension_exact_on_quadratic_stretch():
    # x = s + eps s^2: d/ds [Eh (x_s - 1) x_s] = Eh (2 eps + 8 eps^2 s)
    n, ds, eps, Eh = 15, 0.25, 0.03, 2.5
    s = np.arange(n) * ds
    X = lambda ss: np.stack([ss + eps * ss * ss, 0 * ss, 0 * ss], axis=1)
    gl, gr = _ghosts_from(X, s, ds)
    F = oracle.filament_force(X(s), gl, gr, ds, Eh, 0.0)
    exact = Eh * (2 * eps + 8 * eps * eps * s)
    assert np.allclose(F[1:-1, 0], exact[1:-1], rtol=1e-12, atol=1e-13)
    assert np.abs(F[:, 1:]).max() == 0.0


def test_bending_exact_on_quartic():
    # y = c s^4: -EI d^4y/ds^4 = -24 c EI, exactly for the 4th difference
    n, ds, c, EI = 11, 0.3, 0.02, 0.7
    s = np.arange(n) * ds
    X = lambda ss: np.stack([0 * ss, c * ss ** 4, 0 * ss], axis=1)
    gl, gr = _ghosts_from(X, s, ds)
    F = oracle.filament_force(X(s), gl, gr, ds, 0.0, EI)
    assert np.allclose(F[1:-1, 1], -24 * c * EI, rtol=1e-9)
    assert np.abs(F[:, [0, 2]]).max() == 0.0


# Section 3.1 manufactured solution: L = 1, A = 0.01, E = 0.5 MPa, h = 1 mm;
# readings: rho_s = 1000 kg/m^3 (rho_s h = 1 kg/m^2), EI = E h^3 / 12
A, EH, EI, RHOH = 0.01, 0.5e6 * 1e-3, 0.5e6 * 1e-9 / 12, 1.0


def _mms_X(s, t):
    return np.stack([s, A * np.cos(np.pi * s) * np.sin(np.pi * t), 0 * s], axis=-1)


def _mms_forcing(s, t):
    """B = rho h X_tt - d/ds (T X_s) + EI X_ssss for the manufactured X."""
    ps, pt = np.pi * s, np.pi * t
    ys = -A * np.pi * np.sin(ps) * np.sin(pt)
    yss = -A * np.pi ** 2 * np.cos(ps) * np.sin(pt)
    yssss = A * np.pi ** 4 * np.cos(ps) * np.sin(pt)
    ytt = -A * np.pi ** 2 * np.cos(ps) * np.sin(pt)
    m = np.sqrt(1 + ys * ys)
    T = EH * (m - 1)
    Ts = EH * ys * yss / m
    Bx = -Ts
    By = RHOH * ytt - (Ts * ys + T * yss) + EI * yssss
    return np.stack([Bx, By, 0 * s], axis=-1)


def _mms_error(N, dt, steps, every=50):
    ds = 1.0 / N
    s = np.arange(N + 1) * ds
    Xm, X = _mms_X(s, -dt), _mms_X(s, 0.0)
    err = 0.0
    for n in range(steps):
        t = n * dt
        gl, gr = _mms_X(np.array([-ds]), t)[0], _mms_X(np.array([1 + ds]), t)[0]
        acc = (oracle.filament_force(X, gl, gr, ds, EH, EI) + _mms_forcing(s, t)) / RHOH
        Xn = 2 * X - Xm + dt * dt * acc
        Xn[[0, -1]] = _mms_X(s[[0, -1]], t + dt)
        Xm, X = X, Xn
        if n % every == every - 1:
            err = max(err, np.abs(X - _mms_X(s, t + dt)).max())
    return err


def test_mms_at_the_papers_setup_is_second_order():
    # the paper's own run (Section 3.1): N = 25, 50, 100 elements, dt = 1e-5 s,
    # 1e5 steps, the largest error over all nodes and every step
    ex = golden_fixtures.load("mms_filament_section3_1.txt")
    assert (ex["A_m"], ex["L_m"]) == (A, 1.0)
    assert ex["E_Pa"] * ex["h_m"] == pytest.approx(EH, rel=1e-15)
    assert ex["E_Pa"] * ex["h_m"] ** 3 / 12 == pytest.approx(EI, rel=1e-15)
    Ns = [ex["N_coarsest"] * 2 ** k for k in range(ex["N_refinements"])]
    errs = [_mms_error(N, ex["dt_s"], ex["steps"], every=1) for N in Ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(r - ex["expected_order"]) < 0.1 for r in rates), (errs, rates)


def test_mms_second_order_in_space():
    dt, steps = 1e-5, 20000          # to t = 0.2 s (the ramp-up of the motion)
    errs = [_mms_error(N, dt, steps) for N in (10, 20, 40)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.85 < r < 2.15 for r in rates), (errs, rates)


def test_pretensioned_filament_sine_mode_on_the_lattice():
    # nodes along z at unit spacing, reference ds = 0.9 (stretch 1/0.9),
    # penalty off (alpha = beta = 0): pure filament dynamics inside the
    # oracle's wall-node update
    nz, n, ds, Eh, EI, ms = 44, 37, 0.9, 0.05, 0.01, 1.0
    node = geometry.closed_box(10, 10, nz)
    z = 3.0 + np.arange(n)
    X0 = np.stack([np.full(n, 5.0), np.full(n, 5.0), z], axis=1)
    pinned = np.zeros(n, np.uint8)
    pinned[[0, -1]] = 1
    ib = IBNodes(X0=X0, dA=np.ones(n), ks=np.zeros(n), pinned=pinned, alpha=0.0, beta=0.0, ms=ms,
                 filaments=[np.arange(n)], fil_par=np.array([[ds, Eh, EI]]))
    o = oracle.Oracle(Instance(node=node, tau=0.8, ib=ib))
    amp, k = 1e-4, 1
    th = k * np.pi / (n - 1)
    y0 = amp * np.sin(th * np.arange(n))
    X = X0.copy()
    X[:, 0] += y0
    o.set_ib_state(X, np.zeros_like(X))
    T0 = Eh * (1.0 / ds - 1.0)
    mu = (T0 * 4 * np.sin(th / 2) ** 2 / ds ** 2 + EI * 16 * np.sin(th / 2) ** 4 / ds ** 4) / ms
    om = np.arccos(1 - mu / 2)
    for m in range(1, 201):
        o.step(1)
        got = o.ib_state()[0][:, 0] - 5.0
        want = y0 * (np.cos(om * m) - np.tan(om / 2) * np.sin(om * m))
        assert np.abs(got - want).max() < 1e-3 * amp + 1e-12, m
    # the filament only moves sideways: z stays, the ends stay
    Xe = o.ib_state()[0]
    assert np.abs(Xe[:, 2] - z).max() < 1e-9 and np.all(Xe[[0, -1]] == X[[0, -1]])
