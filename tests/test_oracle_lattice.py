"""Pins of the oracle's lattice update: collision, streaming, halfway
bounce-back, body forcing, boundary flux and non-equilibrium extrapolation.

The references are conservation laws and closed-form flows: mass and
momentum balance, the parabolic channel flow (exact for BGK with halfway
bounce-back at tau = 1/2 + sqrt(3/16)), Hagen-Poiseuille, the planar
Womersley solution, and the identity Eq. Non-equilibrium3 reduces to when
the neighbouring fluid node is in equilibrium.
"""
import numpy as np
import pytest

import oracle
from workloads import BC_RCR, BC_VELOCITY, Boundary, Instance, configs, geometry, profiles

CS2 = 1.0 / 3.0
TAU_MAGIC = 0.5 + np.sqrt(3.0 / 16.0)


def _nu(tau):
    return CS2 * (tau - 0.5)


def test_mass_conserved_closed_box():
    node = geometry.closed_box(8, 9, 10)
    inst = Instance(node=node, tau=0.7)
    o = oracle.Oracle(inst)
    o.set_populations(configs.random_populations(inst, 1, 1e-2))
    fl = node.reshape(-1) == 0
    m0 = o.populations()[:, fl].sum()
    o.step(1000)
    m1 = o.populations()[:, fl].sum()
    assert abs(m1 - m0) / m0 < 1e-12


def test_momentum_balance_periodic_box(d3q19):
    # fully periodic: mass conserved, total momentum grows by exactly N g per step
    node = np.zeros((5, 4, 6), dtype=np.uint8)
    inst = Instance(node=node, tau=0.9)
    o = oracle.Oracle(inst, periodic=7)
    o.set_populations(configs.random_populations(inst, 2, 1e-2))
    f0 = o.populations()
    m0, p0 = f0.sum(), d3q19.T @ f0.sum(axis=1)
    g = np.array([1e-5, -2e-5, 3e-5])
    o.set_body_force(g)
    o.step(50)
    f1 = o.populations()
    N = node.size
    assert abs(f1.sum() - m0) / m0 < 1e-13
    assert np.allclose(d3q19.T @ f1.sum(axis=1), p0 + 50 * N * g, rtol=1e-10, atol=1e-14)


def _channel(tau, ny=10, g=1e-6, steps=20000):
    node = geometry.plates_channel(1, ny, 1)
    o = oracle.Oracle(Instance(node=node, tau=tau), periodic=1 | 4)
    o.set_body_force([g, 0, 0])
    o.step(steps)
    P, jx, jy, jz = o.macros()
    u = jx.reshape(ny) + g / 2
    y = np.arange(ny) + 0.5
    ana = g / (2 * _nu(tau)) * (y - 1.0) * (ny - 1.0 - y)   # walls halfway, at y = 1 and ny - 1
    return y[1:-1], u[1:-1], ana[1:-1]


@pytest.mark.parametrize("tau", [TAU_MAGIC, 0.8, 1.2])
def test_channel_profile_is_parabola(tau):
    y, u, ana = _channel(tau)
    c = np.polyfit(y, u, 2)
    assert np.abs(np.polyval(c, y) - u).max() / u.max() < 1e-10
    assert c[0] == pytest.approx(-1e-6 / (2 * _nu(tau)), rel=1e-8)   # curvature set by g / nu


def test_channel_exact_at_magic_tau():
    y, u, ana = _channel(TAU_MAGIC)
    assert np.abs(u - ana).max() / ana.max() < 1e-9
    y, u, ana = _channel(0.8)
    assert np.abs(u - ana).max() / ana.max() > 1e-3   # a slip elsewhere, as expected for BGK


@pytest.mark.parametrize("R", [4, 6, 8])
def test_tube_hagen_poiseuille(R):
    n = 2 * R + 4
    node = geometry.periodic_tube(n, n, 1, R)
    o = oracle.Oracle(Instance(node=node, tau=TAU_MAGIC), periodic=4)
    g = 1e-6
    o.set_body_force([0, 0, g])
    o.step(int(6 * R * R / _nu(TAU_MAGIC)))
    fl = node.reshape(-1) == 0
    Q = (o.macros()[3][fl] + g / 2).sum()
    R_eff = np.sqrt(fl.sum() / np.pi)     # radius of the staircase cross-section's area
    assert Q == pytest.approx(np.pi * g * R_eff ** 4 / (8 * _nu(TAU_MAGIC)), rel=0.05)


def test_planar_womersley_second_order():
    errs = []
    for ny, T in ((10, 125), (18, 500), (34, 2000)):          # diffusive scaling, alpha fixed
        node = geometry.plates_channel(1, ny, 1)
        o = oracle.Oracle(Instance(node=node, tau=TAU_MAGIC), periodic=1 | 4)
        g0, w, nu = 1e-6, 2 * np.pi / T, _nu(TAU_MAGIC)
        y = np.arange(ny) + 0.5
        k = np.sqrt(1j * w / nu)
        U = g0 / (1j * w) * (1 - np.cosh(k * (y - ny / 2)) / np.cosh(k * (ny - 2) / 2))
        err = mx = 0.0
        for n in range(6 * T):
            b = g0 * np.cos(w * n)
            o.set_body_force([b, 0, 0])
            if n >= 5 * T and n % 5 == 0:
                u = o.macros()[1].reshape(ny)[1:-1] + b / 2
                ua = (U * np.exp(1j * w * n)).real[1:-1]
                err, mx = max(err, np.abs(u - ua).max()), max(mx, np.abs(ua).max())
            o.step(1)
        errs.append(err / mx)
    assert errs[0] < 5e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_flux_of_uniform_flow():
    # f(t_0) = f^eq(P_ref, u e_z) everywhere: the boundary flow fed to the 0D
    # models is the area-mean velocity u, positive into the domain (inlet +u,
    # outlet -u), with the mean gauge pressure 0
    inst = configs.pressure_tube(12, 12, 10, 4.0, 0.8, 0.0, 0.0)
    o = oracle.Oracle(inst)
    N = o.N
    feq = oracle.feq(CS2, [0, 0, 0.01])
    o.set_populations(np.repeat(feq[:, None], N, axis=1))
    o.step(1)
    w = o.waves()[0]
    assert w[1] == pytest.approx(0.01, rel=1e-13) and w[5] == pytest.approx(-0.01, rel=1e-13)
    assert abs(w[2]) < 1e-15 and abs(w[6]) < 1e-15
    s = o.state_0d(0)
    assert s[1] == pytest.approx(0.01 * o.n_xf(0), rel=1e-13)   # literal Q = sum over the layer


def test_nee_equilibrium_neighbour_identity():
    # with x_f in equilibrium and no force, Eq. Non-equilibrium3 gives
    # f_i(x_f, t_1) = f^eq_i(P*, v*) for every population entering from dOmega_2
    v0 = np.array([0.0, 0.0, 0.02])
    p_in, p_out = 3e-3, -2e-3
    inst = configs.pressure_tube(12, 12, 10, 4.0, 0.8, p_in, p_out)
    o = oracle.Oracle(inst)
    feq0 = oracle.feq(CS2, v0)
    o.set_populations(np.repeat(feq0[:, None], o.N, axis=1))
    o.step(1)
    f = o.populations()
    nx, ny, nz = inst.shape
    fin = oracle.feq(CS2 + p_in, v0)
    fout = oracle.feq(CS2 + p_out, v0)
    node = inst.node
    up = [5, 11, 14, 15, 18]      # directions with e_z = +1 in the documented order
    dn = [6, 12, 13, 16, 17]      # e_z = -1
    checked = 0
    for y in range(ny):
        for x in range(nx):
            for i in up:
                ex, ey = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0][i], \
                         [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1][i]
                if node[1, y, x] == 0 and 0 <= x - ex < nx and 0 <= y - ey < ny and node[0, y - ey, x - ex] == 2:
                    assert f[i, x + nx * (y + ny * 1)] == pytest.approx(fin[i], rel=1e-14)
                    checked += 1
            for i in dn:
                ex, ey = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0][i], \
                         [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1][i]
                if node[nz - 2, y, x] == 0 and 0 <= x - ex < nx and 0 <= y - ey < ny and node[nz - 1, y - ey, x - ex] == 3:
                    assert f[i, x + nx * (y + ny * (nz - 2))] == pytest.approx(fout[i], rel=1e-14)
                    checked += 1
    assert checked == o.n_links(0) + o.n_links(1)


def test_pressure_driven_tube_matches_force_driven():
    # Poiseuille flow between two constant-pressure ends coupled by Eq.
    # Non-equilibrium3: the interior pressure is linear, and the cross-section
    # velocity equals the body-force-driven flow with g = -dP/dz
    R, nz, dp = 4, 24, 1e-4
    n = 2 * R + 4
    o = oracle.Oracle(configs.pressure_tube(n, n, nz, R, TAU_MAGIC, dp / 2, -dp / 2))
    o.step(1600)
    P, jx, jy, jz = o.macros()
    Pc = P.reshape(nz, n, n)[:, n // 2, n // 2]
    zz = np.arange(4, nz - 4)
    c = np.polyfit(zz, Pc[4:nz - 4], 1)
    assert np.abs(np.polyval(c, zz) - Pc[4:nz - 4]).max() < 2e-3 * dp
    g = -(Pc[nz // 2 + 4] - Pc[nz // 2 - 4]) / 8.0       # interior gradient at mid-length
    node2 = geometry.periodic_tube(n, n, 1, R)
    o2 = oracle.Oracle(Instance(node=node2, tau=TAU_MAGIC), periodic=4)
    o2.set_body_force([0, 0, g])
    o2.step(1600)
    m = node2[0] == 0
    u1 = jz.reshape(nz, n, n)[nz // 2][m]
    u2 = o2.macros()[3].reshape(n, n)[m] + g / 2
    assert np.abs(u1 - u2).max() / u2.max() < 1e-3
    w = o.waves()[-1]
    assert abs(w[1] + w[5]) / w[1] < 1e-3               # steady: inflow = outflow


def test_velocity_inlet_mass_balance():
    # prescribed plug inflow at the inlet, RCR outlet.  At steady state the
    # momentum density n.j integrated over the inlet layer equals that over the
    # outlet layer (mass balance; Q_u = n.j / sum f, sum f = P / c_s^2), the
    # plug is slowed only by the no-slip rim, and the Windkessel chamber
    # settles at P_w = R_d Q_out.
    nx = ny = 12
    inst = configs.pressure_tube(nx, ny, 16, 4.0, 0.8, 0.0, 0.0)
    u = 0.005
    n_in = inst.boundary_nodes(0).size
    inst.boundaries[0] = Boundary(BC_VELOCITY, 2, +1, [0.0], profile=profiles.plug_profile(n_in, u))
    inst.boundaries[1] = Boundary(BC_RCR, 2, -1, [0.05, 20.0, 1.0, 0.0])
    o = oracle.Oracle(inst)
    o.step(3000)
    w = o.waves()[-1]
    j_in = w[1] * (1 + w[2] / CS2)
    j_out = -w[5] * (1 + w[6] / CS2)
    assert j_in == pytest.approx(j_out, rel=2e-3)      # layer means of a ratio: approximate
    assert 0.7 * u < w[1] < u
    s = o.state_0d(1)
    assert s[4] == pytest.approx(-1.0 * w[5], rel=1e-9)      # P_w = R_d Q_out at steady state


def test_lv_inlet_hybrid_switching_in_lattice():
    # the hybrid ODE-Dirichlet inlet in a small tube: after start-up the valve
    # opens and closes once per beat; while open the inlet pressure follows the
    # ventricular pressure (Section 3.2: inlet and LV pressure coincide in
    # systole); after closure the smoothed Dirichlet condition brings the
    # inflow to zero within N_S steps
    T = 600
    inst = configs.lv_tube(period=T)
    o = oracle.Oracle(inst)
    o.step(5 * T)
    w = o.waves()
    op = w[:, 4]
    opens = np.flatnonzero(np.diff(op) > 0) + 1
    closes = np.flatnonzero(np.diff(op) < 0) + 1
    for beat in (3, 4):
        lo, hi = beat * T, (beat + 1) * T
        assert ((opens >= lo) & (opens < hi)).sum() == 1
        assert ((closes >= lo) & (closes < hi)).sum() == 1
    sl = slice(3 * T, 5 * T)
    Pin, Pv, Qin, opn = w[sl, 2], w[sl, 3], w[sl, 1], w[sl, 4] == 1
    assert np.abs(Pin[opn] - Pv[opn]).max() < 0.1 * Pv.max()
    n_s = int(inst.boundaries[0].params[2])
    c = closes[closes >= 3 * T][0]
    assert np.abs(w[c + n_s + 5: c + n_s + 50, 1]).max() < 0.05 * Qin.max()


@pytest.mark.parametrize("tau", [TAU_MAGIC, 0.8])
def test_wall_shear_channel(tau):
    # steady channel flow: the tangential traction at the first fluid node
    # equals rho nu du/dy there, in the flow direction at both walls; at the
    # magic tau the discrete profile is the analytic parabola, so the value
    # is g (H - 1) / 2 (H = ny - 2); elsewhere it is the slope of the
    # discrete parabola fitted to the node velocities
    ny, g = 12, 1e-6
    node = geometry.plates_channel(1, ny, 1)
    o = oracle.Oracle(Instance(node=node, tau=tau), periodic=1 | 4)
    o.set_body_force([g, 0, 0])
    o.step(40000)
    w = o.wall_shear().reshape(ny, 3)
    u = o.macros()[1].reshape(ny) + g / 2
    y = np.arange(ny) + 0.5
    c = np.polyfit(y[1:-1], u[1:-1], 2)
    slope = np.polyval(np.polyder(c), 1.5)
    nu = _nu(tau)
    assert w[1, 0] == pytest.approx(nu * slope, rel=1e-8)
    assert w[ny - 2, 0] == pytest.approx(w[1, 0], rel=1e-10)         # both walls, along +x
    assert np.abs(w[1, 1:]).max() < 1e-18 and np.abs(w[2:ny - 2]).max() == 0.0
    if tau == TAU_MAGIC:
        assert w[1, 0] == pytest.approx(g * (ny - 3) / 2, rel=1e-9)


def test_wall_shear_tube_direction_and_balance():
    # periodic tube with axial force: the wall traction points along +z and
    # its total over the wall cells balances the body force on the fluid to
    # within the staircase error
    R, g = 6, 1e-6
    n = 2 * R + 4
    node = geometry.periodic_tube(n, n, 1, R)
    o = oracle.Oracle(Instance(node=node, tau=TAU_MAGIC), periodic=4)
    o.set_body_force([0, 0, g])
    o.step(int(6 * R * R / _nu(TAU_MAGIC)))
    w = o.wall_shear()
    at = np.abs(w).sum(axis=1) > 0
    assert at.sum() > 0 and (w[at, 2] > 0).all()
    assert np.abs(w[at, :2]).max() < 0.05 * w[at, 2].max()
    perimeter = 2 * np.pi * R
    mean_wss = g * (node == 0).sum() / perimeter      # force balance per unit length
    assert w[at, 2].mean() == pytest.approx(mean_wss, rel=0.25)


def test_wall_shear_of_uniformly_accelerated_fluid_is_zero():
    # A uniform fluid under a uniform force b accelerates without velocity
    # gradients, so it carries no viscous stress.  Under the BGK update with
    # Guo forcing the non-equilibrium second moment of such a state tends to
    # -(v b + b v)/2 exactly (the recursion Pi_{n+1} = (1 - 1/tau) Pi_n
    # - (v_n b + b v_n)/(2 tau) - b b with v_{n+1} = v_n + b has that particular
    # solution; the start-up decays as (1 - 1/tau)^n), which the (v b + b v)/2
    # term of the stress cancels.  The state is made by the oracle on a fully
    # periodic box, then read out next to the walls of a channel (the wall
    # normal only picks the traction's direction); b has a wall-normal part
    # and v a tangential one, so the term has a tangential traction
    # (1 - 1/(2 tau)) (v_t b_n) / 2 that the read-out must cancel.
    nx, ny, nz, tau = 4, 7, 5, 0.8
    g = np.array([4e-5, 1e-4, -3e-5])
    v0 = np.array([0.03, 0.0, 0.01])
    box = oracle.Oracle(Instance(node=np.zeros((nz, ny, nx), np.uint8), tau=tau), periodic=7)
    box.set_body_force(g)
    box.set_populations(np.repeat(oracle.feq(CS2, v0)[:, None], nx * ny * nz, axis=1))
    box.step(80)
    f = box.populations()
    assert np.abs(f - f[:, :1]).max() == 0.0                 # still uniform
    node = geometry.plates_channel(nx, ny, nz)                 # walls at y = 0 and y = ny - 1
    ch = oracle.Oracle(Instance(node=node, tau=tau), periodic=1 | 4)
    ch.set_populations(f)
    ch.set_body_force(g)
    w = ch.wall_shear().reshape(nz, ny, nx, 3)
    v = box.macros()[1:]
    vx, vz = v[0][0] + g[0] / 2, v[2][0] + g[2] / 2
    term = (1 - 1 / (2 * tau)) * 0.5 * np.array([vx * g[1], vz * g[1]])   # what a missing term leaves
    assert np.abs(term).min() > 1e-7
    assert np.abs(w[:, [1, ny - 2]]).max() < 1e-9 * np.abs(term).max()
    assert np.abs(w[:, 2:ny - 2]).max() == 0.0


def test_nee_copies_the_neighbours_non_equilibrium():
    # Eq. Non-equilibrium3 with a pressure-type 0D node and x_f out of
    # equilibrium: the population entering x_f from the node is
    # f*_i(x_f) + f^eq_i(P*, v(x_f)) - f^eq_i(P(x_f), v(x_f)), i.e. the
    # neighbour's post-collision population shifted by w_i (P* - P(x_f)) / c_s^2.
    # f^eq (Eq. feq, rho0 = 1) and the BGK step are restated here.
    ex = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    ey = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    ez = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)

    def feq(P, v):
        eu = ex * v[0] + ey * v[1] + ez * v[2]
        return w * (P / CS2 + 3 * eu + 4.5 * eu * eu - 1.5 * (v @ v))

    tau, p_in, p_out = 0.8, 3e-3, -2e-3
    inst = configs.pressure_tube(12, 12, 10, 4.0, tau, p_in, p_out)
    f0 = configs.random_populations(inst, seed=11, amp=2e-2)
    o = oracle.Oracle(inst)
    o.set_populations(f0)
    o.step(1)
    f1 = o.populations()
    nx, ny, nz = inst.shape
    node = inst.node
    checked = 0
    for z_f, z_b, code, p0d, dirs in ((1, 0, 2, p_in, np.flatnonzero(ez == 1)),
                                       (nz - 2, nz - 1, 3, p_out, np.flatnonzero(ez == -1))):
        for y in range(ny):
            for x in range(nx):
                if node[z_f, y, x] != 0:
                    continue
                c = x + nx * (y + ny * z_f)
                f = f0[:, c]
                P = CS2 * f.sum()
                v = np.array([ex @ f, ey @ f, ez @ f])
                fstar = f - (f - feq(P, v)) / tau
                for i in dirs:
                    xb, yb = x - ex[i], y - ey[i]
                    if not (0 <= xb < nx and 0 <= yb < ny) or node[z_b, yb, xb] != code:
                        continue
                    want = fstar[i] + feq(CS2 + p0d, v)[i] - feq(P, v)[i]
                    assert f1[i, c] == pytest.approx(want, rel=1e-13, abs=1e-16)
                    # the pressure form of the same identity
                    assert want == pytest.approx(fstar[i] + w[i] * (CS2 + p0d - P) / CS2, rel=1e-13)
                    checked += 1
    assert checked == o.n_links(0) + o.n_links(1) > 0


def test_velocity_inlet_prescribes_the_next_steps_value():
    # Algorithm 1 sets the 0D value of t_{n+1} before the coupling of that
    # step: from rest (x_f at equilibrium), the population entering x_f from
    # an inlet node after step 0 -> 1 is f^eq_i(P(x_f), v*(t_1)) with
    # v* = u_mean + Re{c e^{i omega t}} of that node (Eq. Non-equilibrium3,
    # velocity type), here along +z.  f^eq (Eq. feq, rho0 = 1) is restated.
    ex = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    ey = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    ez = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    inst = configs.rigid_tube(12, 12, 10, radius=4.0, period=40)   # a short beat: v* moves fast
    omega = inst.boundaries[0].params[0]
    prof = inst.boundaries[0].profile
    nx, ny, nz = inst.shape
    nodes = inst.boundary_nodes(0)
    o = oracle.Oracle(inst)
    o.set_populations(np.repeat(w[:, None], o.N, axis=1))   # rest: P = c_s^2, v = 0
    o.step(1)
    f1 = o.populations()
    checked = 0
    for q, b in enumerate(nodes):
        xb, yb = b % nx, (b // nx) % ny
        vz = prof[q, 0] + prof[q, 1] * np.cos(omega * 1.0) - prof[q, 2] * np.sin(omega * 1.0)
        for i in np.flatnonzero(ez == 1):
            x, y = xb + ex[i], yb + ey[i]
            if not (0 <= x < nx and 0 <= y < ny) or inst.node[1, y, x] != 0:
                continue
            want = w[i] * (1.0 + 3 * vz + 4.5 * vz * vz - 1.5 * vz * vz)
            assert f1[i, x + nx * (y + ny * 1)] == pytest.approx(want, rel=1e-13)
            checked += 1
    assert checked == o.n_links(0) > 0
    # the value of t_0 would differ by far more than the tolerance
    assert abs(np.cos(omega) - 1.0) > 1e-3


def test_nee_carries_the_neighbours_forcing():
    # Eq. Non-equilibrium3 rests on f*_i(x_f) = f^eq_i + (1 - 1/tau) f^neq_i + F_i:
    # with a force density b at x_f the entering population is the neighbour's
    # forced post-collision value, shifted by f^eq_i(P*, v) - f^eq_i(P(x_f), v),
    # v = j + b/2 (Eq. v).  f^eq (Eq. feq), Guo's F_i (Eq. f) and the BGK step
    # are restated here.
    ex = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    ey = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    ez = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    E = np.stack([ex, ey, ez], axis=1).astype(float)

    def feq(P, v):
        eu = E @ v
        return w * (P / CS2 + 3 * eu + 4.5 * eu * eu - 1.5 * (v @ v))

    def guo(tau, v, b):
        eu, eb = E @ v, E @ b
        return (1 - 0.5 / tau) * w * (3 * (eb - v @ b) + 9 * eu * eb)

    tau, p_in, p_out = 0.8, 3e-3, -2e-3
    g = np.array([2e-4, -1e-4, 3e-4])
    inst = configs.pressure_tube(12, 12, 10, 4.0, tau, p_in, p_out)
    f0 = configs.random_populations(inst, seed=5, amp=1e-2)
    o = oracle.Oracle(inst)
    o.set_populations(f0)
    o.set_body_force(list(g))
    o.step(1)
    f1 = o.populations()
    nx, ny, nz = inst.shape
    node = inst.node
    checked, shift = 0, 0.0
    for z_f, z_b, code, p0d, dirs in ((1, 0, 2, p_in, np.flatnonzero(ez == 1)),
                                       (nz - 2, nz - 1, 3, p_out, np.flatnonzero(ez == -1))):
        for y in range(ny):
            for x in range(nx):
                if node[z_f, y, x] != 0:
                    continue
                c = x + nx * (y + ny * z_f)
                f = f0[:, c]
                P = CS2 * f.sum()
                v = E.T @ f + g / 2
                fstar = f - (f - feq(P, v)) / tau + guo(tau, v, g)
                for i in dirs:
                    xb, yb = x - ex[i], y - ey[i]
                    if not (0 <= xb < nx and 0 <= yb < ny) or node[z_b, yb, xb] != code:
                        continue
                    want = fstar[i] + feq(CS2 + p0d, v)[i] - feq(P, v)[i]
                    assert f1[i, c] == pytest.approx(want, rel=1e-13, abs=1e-16)
                    shift = max(shift, abs(guo(tau, v, g)[i]))
                    checked += 1
    assert checked == o.n_links(0) + o.n_links(1) > 0
    assert shift > 1e-6   # the forcing term is far above the tolerance


def test_closed_valve_velocity_is_smoothed_at_the_next_steps_time():
    # after the aortic valve closes in the step from t_n (T_d = t_n), the inlet
    # links prescribe v* = v_0(T_d) S(t_{m+1}, T_d, N_S) in every later step m
    # (Eqs. SmoothFunction, vnew; the 0D value of t_{m+1} as Algorithm 1 orders
    # it), with v_0 the closure-step velocity of each link's x_f and P* = P(x_f):
    # the entering population is f^eq(P(x_f), v*) + (1 - 1/tau) f^neq(x_f).
    # f^eq (Eq. feq) and S (Eq. SmoothFunction) are restated here.
    ex = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    ey = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    ez = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    E = np.stack([ex, ey, ez], axis=1).astype(float)

    def feq(P, v):
        eu = E @ v
        return w * (P / CS2 + 3 * eu + 4.5 * eu * eu - 1.5 * (v @ v))

    def S(t, t0, L):
        if t <= t0:
            return 1.0
        if t >= t0 + L:
            return 0.0
        u = (t - t0) / L
        return float(np.exp(2.0 * np.exp(-1.0 / u) / (u - 1.0)))

    inst = configs.lv_tube(period=300)
    tau, n_s = inst.tau, inst.boundaries[0].params[2]
    nx, ny, nz = inst.shape
    o = oracle.Oracle(inst)
    links = []
    for y in range(ny):
        for x in range(nx):
            if inst.node[1, y, x] != 0:
                continue
            for i in np.flatnonzero(ez == 1):
                xb, yb = x - ex[i], y - ey[i]
                if 0 <= xb < nx and 0 <= yb < ny and inst.node[0, yb, xb] == 2:
                    links.append((x + nx * (y + ny * 1), i))
    assert len(links) == o.n_links(0)
    was_open, Td, v0, checked = 0.0, None, {}, 0
    for n in range(1200):
        f = o.populations()
        o.step(1)
        st = o.state_0d(0)
        if Td is None and was_open == 1.0 and st[6] == 0.0:
            Td = n
            assert st[7] == pytest.approx(Td)
            v0 = {c: E.T @ f[:, c] for c, _ in links}           # no force here: v = j
        was_open = st[6]
        if Td is not None and n in (Td, Td + 1, Td + n_s // 2) and st[6] == 0.0:
            f1 = o.populations()
            s = S(n + 1.0, Td, n_s)
            for c, i in links:
                P, v = CS2 * f[:, c].sum(), E.T @ f[:, c]
                want = feq(P, v0[c] * s)[i] + (1 - 1 / tau) * (f[i, c] - feq(P, v)[i])
                assert f1[i, c] == pytest.approx(want, rel=1e-12, abs=1e-15), (n, Td, i)
                checked += 1
            if n == Td + n_s // 2:
                break
    assert Td is not None and checked == 3 * len(links)
    # one step earlier the smoothing factor differs far beyond the tolerance
    assert abs(S(Td + n_s / 2 + 1, Td, n_s) - S(Td + n_s / 2, Td, n_s)) > 1e-3
