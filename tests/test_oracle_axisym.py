"""Pins of the axisymmetric D2Q9 oracle (Section 2.3.1, Eq. Afi with the
axisymmetric source; readings in oracle/axisym.py) against closed forms of
axisymmetric pipe flow.

* a fluid at rest stays at rest exactly;
* steady Hagen-Poiseuille flow u = G (R^2 - r^2) / (4 nu) in a periodic pipe,
  second order in R (the planar lattice alone would give twice that);
* Womersley flow (J0 profile) under an oscillating axial force, second order
  under diffusive scaling;
* mass: through a stenosis between a velocity inlet and a pressure outlet
  the flow rate 2 pi sum r u_x is the same at every cross-section to the
  staircase error; with the mass source planted out it is not;
* the hybrid LV inlet opens and closes once per beat on the axisymmetric
  tube.
"""
import numpy as np
import pytest
from scipy import special

import oracle.axisym as ax
from workloads import axisym as axw
from workloads.spec import BC_PRESSURE, BC_VELOCITY, Boundary


def test_rest_stays_at_rest():
    node, _ = axw.stenosis(10, 24, 8.0, 3.0, 5.0)
    o = ax.AxiOracle(node, 0.7, [Boundary(BC_PRESSURE, 0, +1, [0.0]), Boundary(BC_PRESSURE, 0, -1, [0.0])])
    o.step(50)
    P, ux, ur = o.fields()
    fl = o.fluid
    assert np.abs(P[fl] - ax.PREF).max() < 1e-15 and np.abs(ux).max() < 1e-15 and np.abs(ur).max() < 1e-15


def test_hagen_poiseuille_second_order():
    tau, G = 0.8, 1e-6
    nu = (tau - 0.5) / 3
    errs = []
    for R in (5, 10, 20):
        o = ax.AxiOracle(np.zeros((R, 1), np.uint8), tau, periodic_x=True, body_force=G)
        o.step(int(6 * R * R / nu))
        r = np.arange(R) + 0.5
        ua = G / (4 * nu) * (R * R - r * r)
        errs.append(np.abs(o.fields()[1][:, 0] - ua).max() / ua.max())
    assert errs[0] < 6e-3
    assert all(3.8 < errs[i] / errs[i + 1] < 4.2 for i in range(2)), errs


def test_womersley_second_order():
    tau, G0, alpha = 0.8, 1e-6, 3.0
    nu = (tau - 0.5) / 3
    i32 = np.exp(0.75j * np.pi)
    errs = []
    for R in (4, 8, 16):
        w = (alpha / R) ** 2 * nu
        T = 2 * np.pi / w
        o = ax.AxiOracle(np.zeros((R, 1), np.uint8), tau, periodic_x=True)
        r = np.arange(R) + 0.5
        U = G0 / (1j * w) * (1 - special.jv(0, i32 * alpha * r / R) / special.jv(0, i32 * alpha))
        err = mx = 0.0
        for n in range(int(5 * T)):
            o.Gx = G0 * np.cos(w * n)
            o.step(1)
            if n > 4 * T:
                o.Gx = G0 * np.cos(w * (n + 1))
                ua = (U * np.exp(1j * w * (n + 1))).real
                err = max(err, np.abs(o.fields()[1][:, 0] - ua).max())
                mx = max(mx, np.abs(ua).max())
        errs.append(err / mx)
    assert errs[0] < 2e-2
    assert errs[0] / errs[1] > 3.2 and errs[1] / errs[2] > 3.5, errs


def _stenosis_flux_spread(plant_no_mass_source: bool):
    node, _ = axw.stenosis(12, 64, 10.0, 4.0, 8.0)
    n_in = int((node[:, 0] == 2).sum())
    r = np.arange(n_in) + 0.5
    prof = np.zeros((n_in, 3))
    prof[:, 0] = 0.02 * (1 - (r / 10.0) ** 2)
    bcs = [Boundary(BC_VELOCITY, 0, +1, [0.0], profile=prof), Boundary(BC_PRESSURE, 0, -1, [0.0])]
    o = ax.AxiOracle(node, 1.0, bcs)
    if plant_no_mass_source:
        def no_mass(self, _orig=ax.AxiOracle._macros):
            _orig(self)
            self.m[:] = 0.0
            self.P = ax.CS2 * self.sf
        o._macros = no_mass.__get__(o)
    o.step(12000)
    ux = o.fields()[1]
    rr = (np.arange(o.nr) + 0.5)[:, None]
    Q = (2 * np.pi * rr * ux * o.fluid).sum(axis=0)[1:-1]
    return (Q.max() - Q.min()) / Q.mean()


def test_flow_rate_conserved_through_stenosis():
    assert _stenosis_flux_spread(False) < 0.03      # 2.2 %; 0.58 % at twice the resolution
    assert _stenosis_flux_spread(True) > 0.3        # mass source planted out: 43 %


def test_lv_inlet_cycles_on_axisymmetric_tube():
    inst = axw.lv_tube(nr=8, nx=40, period=600)
    o = ax.AxiOracle(inst.node, inst.tau, inst.boundaries)
    o.step(1800)
    w = o.waves()
    valve = w[:, 4]
    opens = int((np.diff(valve) > 0).sum())
    closes = int((np.diff(valve) < 0).sum())
    assert opens >= 2 and closes >= 2
    # while the valve is open the inlet pressure follows the ventricle (pressure-type coupling)
    assert np.abs(w[valve == 1, 2]).max() > 0


def test_straight_aorta_workload_is_the_papers_case():
    # the convergence workload is built on the paper's printed case: 25 diameters,
    # Womersley number 16 at every printed resolution (diffusive scaling keeps it)
    import math

    import golden_fixtures
    from paper_2112_05258_gb300 import e5_study
    from workloads import axisym as wa
    from workloads.configs import viscosity
    ex = golden_fixtures.load("straight_aorta_section3_1_3.txt")
    printed = tuple(ex[f"n_d_{k}"] for k in range(1, 6))
    assert tuple(e5_study.RESOLUTIONS) == printed
    for n_d in printed[:3]:
        inst = wa.straight_aorta(n_d)
        nr, nx = inst.node.shape
        assert nx - 2 == round(ex["length_D"] * n_d)          # lattice length in diameters
        T = wa.e5_period(n_d)
        alpha = (n_d / 2.0) * math.sqrt(2 * math.pi / T / viscosity(inst.tau))
        assert alpha == pytest.approx(ex["womersley"], rel=1e-12)


def _mms_fields(x, r, R, A, k):
    """Manufactured axisymmetric flow from the Stokes stream function
    psi = A r^2 (1 - r^2/R^2)^2 sin(k x): u_x = psi_r / r, u_r = -psi_x / r.
    It is divergence-free in the axisymmetric sense, vanishes on the wall
    r = R, and is regular on the axis (u_r ~ r, d_r u_x = 0)."""
    s = (r / R) ** 2
    ux = 2 * A * np.sin(k * x) * (1 - s) * (1 - 3 * s)
    ur = -A * k * r * (1 - s) ** 2 * np.cos(k * x)
    return ux, ur


def _mms_force(x, r, R, A, k, nu, h=1e-4):
    """Body force that makes the manufactured flow a steady solution of the
    axisymmetric incompressible Navier-Stokes equations with constant
    pressure: g = (u.grad) u - nu lap u, lap of the radial component with
    the -u_r / r^2 term; derivatives by central differences of the closed
    form (step h, error ~h^2)."""
    f = lambda a, b: _mms_fields(a, b, R, A, k)
    u = f(x, r)
    xp, xm, rp, rm = f(x + h, r), f(x - h, r), f(x, r + h), f(x, r - h)
    g = []
    for c in range(2):
        dx = (xp[c] - xm[c]) / (2 * h)
        dr = (rp[c] - rm[c]) / (2 * h)
        lap = (xp[c] - 2 * u[c] + xm[c]) / h ** 2 + (rp[c] - 2 * u[c] + rm[c]) / h ** 2 + dr / r
        if c == 1:
            lap -= u[1] / r ** 2
        g.append(u[0] * dx + u[1] * dr - nu * lap)
    return g


def _mms_error(R, tau=0.8):
    nu = (tau - 0.5) / 3
    nx = 4 * R
    k = 2 * np.pi / nx
    A = 0.16 / R                      # fixed Reynolds number 2 A R / nu = 3.2 under refinement
    x = np.arange(nx)[None, :] * np.ones((R, 1))
    r = (np.arange(R) + 0.5)[:, None] * np.ones((1, nx))
    o = ax.AxiOracle(np.zeros((R, nx), np.uint8), tau, periodic_x=True, body_force=_mms_force(x, r, R, A, k, nu))
    ux, ur = _mms_fields(x, r, R, A, k)
    o.set_populations(ax.feq(ax.CS2 + 0 * ux, ux, ur))
    o.step(int(8 * R * R / nu))       # eight viscous times: steady to far below the error
    _, vx, vr = o.fields()
    um = np.abs(ux).max()
    assert np.abs(ur).max() > 0.2 * um      # a flow with real radial velocity
    return np.abs(vx - ux).max() / um, np.abs(vr - ur).max() / um


def test_manufactured_radial_flow_converges():
    # every source term is active: mass -u_r/r, the viscous terms with d_x u_r
    # and d_r u_r, and the convective -u_x u_r / r and -u_r^2 / r (Reynolds
    # number 3.2, so leaving either out moves the steady flow by percents)
    e8 = _mms_error(8)
    e16 = _mms_error(16)
    assert e16[0] < 8e-3 and e16[1] < 1.5e-3, (e8, e16)
    assert e8[0] / e16[0] > 3.0 and e8[1] / e16[1] > 2.5, (e8, e16)
