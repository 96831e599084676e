"""Pins of the oracle's immersed-boundary exchange (Eqs. LagForce,
interpolation, EulForce) and of the spring wall update.

References: properties of the discrete delta (support, symmetry, partition
of unity), exactness of interpolation where the kernel's first moment
vanishes, total-force conservation of spreading, momentum balance of the
fluid, the feedback sign of the penalty, and the closed-form discrete
oscillator of symplectic Euler.
"""
import numpy as np
import pytest

import oracle
from workloads import IBNodes, Instance, configs

CS2 = 1.0 / 3.0


def test_delta_kernel_properties():
    assert oracle.phi(0.0) == pytest.approx(0.5, abs=1e-16)
    assert oracle.phi(2.0) == 0.0 and oracle.phi(-2.0) == 0.0 and oracle.phi(2.5) == 0.0
    rng = np.random.default_rng(0)
    for th in rng.uniform(0, 1, 50):
        r = np.array([-1 - th, -th, 1 - th, 2 - th])
        assert sum(oracle.phi(x) for x in r) == pytest.approx(1.0, abs=1e-15)
        assert oracle.phi(th) == oracle.phi(-th)
    # first moment vanishes at half-integer offsets
    r = np.array([-1.5, -0.5, 0.5, 1.5])
    assert abs(sum(x * oracle.phi(x) for x in r)) < 1e-16


def _box_with_nodes(X0, alpha=-0.0, beta=-0.0, ks=None, ms=1.0, pinned=None, n=12):
    node = np.zeros((n, n, n), dtype=np.uint8)
    ns = X0.shape[0]
    ib = IBNodes(X0=np.asarray(X0, float), dA=np.ones(ns), ks=np.zeros(ns) if ks is None else ks,
                 pinned=np.zeros(ns, np.uint8) if pinned is None else pinned,
                 alpha=alpha, beta=beta, ms=ms)
    inst = Instance(node=node, tau=0.8, ib=ib)
    return inst, oracle.Oracle(inst, periodic=7)


def _fill_velocity(o, inst, vfun):
    nx, ny, nz = inst.shape
    f = np.empty((19, o.N))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f[:, x + nx * (y + ny * z)] = oracle.feq(CS2, vfun(np.array([x + 0.5, y + 0.5, z + 0.5])))
    o.set_populations(f)


def test_interpolation_of_constant_and_linear_fields():
    rng = np.random.default_rng(1)
    X0 = np.vstack([rng.uniform(4, 8, (6, 3)),                     # generic positions
                    np.array([[5.0, 6.0, 7.0], [6.0, 6.0, 6.0]])])  # integer: cell faces, zero first moment
    inst, o = _box_with_nodes(X0)
    u0 = np.array([0.01, -0.02, 0.005])
    _fill_velocity(o, inst, lambda p: u0)
    o.step(1)
    Vf = o.ib_state()[3]
    assert np.allclose(Vf, u0, atol=1e-16)                  # partition of unity
    G = np.array([[1e-3, 2e-4, 0.0], [0.0, -5e-4, 1e-4], [3e-4, 0.0, 2e-4]])
    inst, o = _box_with_nodes(X0)
    _fill_velocity(o, inst, lambda p: u0 + G @ (p - 6.0))
    o.step(1)
    Vf = o.ib_state()[3]
    # separable kernel: V_f = v(X) + G m1, m1_a = sum_k r_k phi(r_k) along axis a
    for s, X in enumerate(X0):
        m1 = np.empty(3)
        for a in range(3):
            th = (X[a] - 0.5) - np.floor(X[a] - 0.5)
            r = np.array([-1 - th, -th, 1 - th, 2 - th])
            m1[a] = sum(x * oracle.phi(x) for x in r)
        assert np.allclose(Vf[s], u0 + G @ (X - 6.0) + G @ m1, atol=1e-15)
    assert np.allclose(Vf[-2:], [u0 + G @ (X - 6.0) for X in X0[-2:]], atol=1e-16)


def test_spreading_conserves_force_and_momentum(d3q19):
    rng = np.random.default_rng(2)
    X0 = rng.uniform(4, 8, (5, 3))
    inst, o = _box_with_nodes(X0, alpha=-1e-3, beta=-0.5)
    _fill_velocity(o, inst, lambda p: np.array([0.01, 0.0, -0.004]))
    p0 = d3q19.T @ o.populations().sum(axis=1)
    o.step(1)
    bx, by, bz = o.force()
    F = o.ib_state()[2]
    assert np.allclose([bx.sum(), by.sum(), bz.sum()], F.sum(axis=0), rtol=1e-13, atol=1e-18)
    # fluid momentum changes by exactly the spread force (periodic box)
    p1 = d3q19.T @ o.populations().sum(axis=1)
    assert np.allclose(p1 - p0, F.sum(axis=0), rtol=1e-10, atol=1e-16)


def test_penalty_is_a_feedback():
    # a pinned node in a uniform stream: the force on the fluid opposes the
    # slip V_f - V_s, and the fluid near the node slows relative to a run
    # without the wall node
    X0 = np.array([[6.0, 6.0, 6.0]])
    u0 = np.array([0.0, 0.0, 0.01])
    inst, o = _box_with_nodes(X0, alpha=-1e-3, beta=-0.5, pinned=np.ones(1, np.uint8))
    _fill_velocity(o, inst, lambda p: u0)
    o.step(1)
    X, Vs, F, Vf = o.ib_state()
    assert np.dot(F[0], Vf[0] - Vs[0]) < 0
    o.step(20)
    near = 5 + 12 * (5 + 12 * 5)
    inst2, o2 = _box_with_nodes(X0, pinned=np.ones(1, np.uint8))
    _fill_velocity(o2, inst2, lambda p: u0)
    o2.step(21)
    assert o.macros()[3][near] < o2.macros()[3][near]
    assert np.allclose(o.ib_state()[0], X0)                  # pinned node stays at X0


def test_spring_wall_discrete_oscillator():
    # fluid at rest and no coupling (alpha = beta = 0): a node released at
    # X0 + d follows symplectic Euler of m x'' = -k (x - X0), whose closed form
    # is x_n - X0 = d [cos(n th) + c sin(n th)], cos th = 1 - w^2/2,
    # c = -w^2 / (2 sin th), w^2 = k / m
    X0 = np.array([[6.0, 6.0, 6.0], [5.0, 7.0, 6.5]])
    k, m, d = 0.02, 2.0, 0.3
    inst, o = _box_with_nodes(X0, ks=np.array([k, k]), ms=m, pinned=np.array([0, 1], np.uint8))
    o.set_ib_state(X0 + np.array([d, 0.0, 0.0]), np.zeros((2, 3)))
    w2 = k / m
    th = np.arccos(1 - w2 / 2)
    c = -w2 / (2 * np.sin(th))
    for n in range(1, 200):
        o.step(1)
        if n % 37 == 0:
            X = o.ib_state()[0]
            assert X[0, 0] - X0[0, 0] == pytest.approx(d * (np.cos(n * th) + c * np.sin(n * th)), abs=1e-13)
            assert np.allclose(X[0, 1:], X0[0, 1:], atol=1e-15)
            assert np.allclose(X[1], X0[1] + [d, 0, 0])     # pinned: never moves


def test_membrane_motion_stays_bounded():
    # Eq. interpolation samples the fluid velocity of Eq. v (j + b/2); with
    # the unforced j instead, the slip b/2 that the penalty integral cannot
    # see makes the membrane of the Womersley-driven IB tube collapse inward
    # within one beat at a tenfold integral gain (mean radial displacement
    # -0.52 cells after 4000 steps); with Eq. v it oscillates with the beat
    inst = configs.ib_tube()
    inst.ib.alpha = 10 * inst.ib.alpha
    o = oracle.Oracle(inst)
    c = np.array([inst.shape[0] / 2, inst.shape[1] / 2])
    r0 = np.hypot(*(inst.ib.X0[:, :2] - c).T)
    for _ in range(4):
        o.step(1000)
        X = o.ib_state()[0]
        dr = np.hypot(*(X[:, :2] - c).T) - r0
        assert abs(dr.mean()) < 0.03
        assert np.percentile(np.linalg.norm(X - inst.ib.X0, axis=1), 99) < 0.2


def test_interpolated_velocity_includes_half_the_force_density():
    # the IB interpolates the fluid velocity of Eq. v, j/rho0 + b/(2 rho0), of
    # f(t_n) with the force density b still held from the previous step: in a
    # periodic box under a uniform body force g and with the penalty off, b is
    # g after the first step, so the second step's V_f is j(t_1) + g/2 for
    # every node (partition of unity; j summed here from f(t_1))
    rng = np.random.default_rng(3)
    X0 = rng.uniform(4, 8, (6, 3))
    inst, o = _box_with_nodes(X0)
    u0 = np.array([0.01, -0.02, 0.005])
    g = np.array([3e-4, -2e-4, 5e-4])
    _fill_velocity(o, inst, lambda p: u0)
    o.set_body_force(list(g))
    o.step(1)
    f1 = o.populations()
    ex = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    ey = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    ez = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    j1 = np.stack([ex @ f1, ey @ f1, ez @ f1], axis=1)
    assert np.abs(j1 - j1[0]).max() < 1e-15                 # uniform field
    o.step(1)
    Vf = o.ib_state()[3]
    assert np.allclose(Vf, j1[0] + g / 2, rtol=0, atol=1e-15), (Vf[0], j1[0], g)
    assert np.abs(g / 2).min() > 1e-5                        # far above the tolerance
