"""The benchmark workloads as seeded synthetic instances.

* ``rigid_tube``: D3Q19 BGK, tau = 0.8, 24x24x64 box, straight tube of
  radius 8 along z with halfway bounce-back walls; Womersley inlet (peak
  u = 0.02, period 1000 steps); RCR outlet (R_p = 0.05, C = 200, R_d = 1).
* ``aorta``: 128x128x1024 tapered, spline-curved tube (radius 40 -> 24) with
  two radius-10 side branches, LV elastance inlet, RCR outlets and about
  2e5 Lagrangian wall nodes (see :mod:`workloads.aorta`).
* ``tube_batch``: many rigid tubes of uneven sizes (see :mod:`workloads.batch`).
"""
from __future__ import annotations

import numpy as np

from . import geometry, profiles
from .spec import (BC_LV, BC_PRESSURE, BC_RCR, BC_VELOCITY, Boundary,
                   Instance)

CS2 = 1.0 / 3.0


def viscosity(tau: float) -> float:
    """Kinematic viscosity of a BGK lattice in lattice units, c_s^2 (tau - 1/2)."""
    return CS2 * (tau - 0.5)


def rigid_tube(nx: int = 24, ny: int = 24, nz: int = 64, radius: float = 8.0,
               tau: float = 0.8, u_peak: float = 0.02, period: int = 1000,
               rcr=(0.05, 200.0, 1.0, 0.0), q_scale: int = 1,
               inlet_kind: int = BC_VELOCITY) -> Instance:
    """Straight rigid tube, Womersley (or LV) inlet, RCR outlet."""
    node = geometry.straight_tube(nx, ny, nz, radius)
    inst = Instance(node=node, tau=tau, q_scale=q_scale,
                    name=f"rigid_tube_{nx}x{ny}x{nz}_R{radius:g}")
    omega = 2.0 * np.pi / period
    if inlet_kind == BC_VELOCITY:
        r = geometry.node_radius(nx, ny, inst.boundary_nodes(0))
        prof = profiles.womersley_coefficients(r, radius, omega, viscosity(tau), u_peak)
        inst.boundaries.append(Boundary(BC_VELOCITY, 2, +1, [omega], profile=prof))
    elif inlet_kind == BC_LV:
        inst.boundaries.append(lv_boundary(period=period))
    else:
        raise ValueError(inlet_kind)
    inst.boundaries.append(Boundary(BC_RCR, 2, -1, list(rcr)))
    return inst


# Lattice scaling of the ventricular elastance: E_max = 2.0 and E_min = 0.06
# (mmHg/ml in the clinical curve) times KAPPA, with ventricular volume measured
# as the time integral of the area-mean inlet velocity.  With the filling
# pressure P_LA this gives a stroke of about 26 lattice lengths and peak
# ventricular gauge pressure of order 1e-2, well below c_s^2 = 1/3.
LV_KAPPA = 4.9e-4
LV_P_LA = 1.0e-3


def lv_boundary(period: int = 4000, e_max: float = 2.0, e_min: float = 0.06,
                kappa: float = LV_KAPPA, p_la: float = LV_P_LA,
                n_s: int | None = None, axis: int = 2, sign: int = +1) -> Boundary:
    """LV elastance inlet with the double-Hill curve sampled per step.

    N_S defaults to round(0.075 * period), the ratio of the smoothing
    example of Section 2.2.1 (15 steps of 0.005 s in a 1 s beat).
    """
    if n_s is None:
        n_s = int(round(0.075 * period))
    tab = profiles.elastance_table(period, e_max * kappa, e_min * kappa)
    return Boundary(BC_LV, axis, sign, [float(period), p_la, float(n_s), p_la],
                    elastance=tab)


def lv_tube(nx: int = 14, ny: int = 14, nz: int = 32, radius: float = 5.0,
            tau: float = 0.8, period: int = 600) -> Instance:
    """Small rigid tube with the hybrid LV inlet and an RCR outlet.

    The elastance scale grows as the beat shortens (KAPPA * 4000 / period)
    so that the stroke, measured in lattice lengths, stays proportionate to
    the beat; the Windkessel (R_p = 0.02, C = 1200, R_d = 1) keeps the
    diastolic pressure above the atrial pressure so that the valve opens and
    closes once per beat after a short start-up.
    """
    inst = rigid_tube(nx, ny, nz, radius, tau, period=period,
                      rcr=(0.02, 1200.0, 1.0, 0.0), inlet_kind=BC_LV)
    inst.boundaries[0] = lv_boundary(period=period, kappa=LV_KAPPA * 4000.0 / period)
    inst.name = f"lv_tube_{nx}x{ny}x{nz}_R{radius:g}_T{period}"
    return inst


def lv_tube_x(nx: int = 30, ny: int = 12, nz: int = 12, radius: float = 4.3,
              tau: float = 0.8, period: int = 300) -> Instance:
    """The LV tube of :func:`lv_tube` laid along x: inlet plane x = 0, outlet
    plane x = nx - 1, so that every lattice row of the vessel begins and ends
    with a 0D boundary node."""
    z = lv_tube(nx=ny, ny=nz, nz=nx, radius=radius, tau=tau, period=period)
    node = np.ascontiguousarray(z.node.transpose(2, 1, 0))
    inst = Instance(node=node, tau=tau, name=f"lv_tube_x_{nx}x{ny}x{nz}_R{radius:g}_T{period}")
    inst.boundaries.append(lv_boundary(period=period, kappa=LV_KAPPA * 4000.0 / period, axis=0, sign=+1))
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, list(z.boundaries[1].params)))
    return inst


def pressure_tube(nx: int, ny: int, nz: int, radius: float, tau: float,
                  p_in: float, p_out: float) -> Instance:
    """Tube driven by two constant-pressure ends (NEE pressure coupling)."""
    node = geometry.straight_tube(nx, ny, nz, radius)
    inst = Instance(node=node, tau=tau, name="pressure_tube")
    inst.boundaries.append(Boundary(BC_PRESSURE, 2, +1, [p_in]))
    inst.boundaries.append(Boundary(BC_PRESSURE, 2, -1, [p_out]))
    return inst


def random_populations(inst: Instance, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Seeded initial populations f_i(x, t_0) = w_i (1 + amp * U[-1, 1]).

    Returned as ``(19, nz*ny*nx)`` float64 in the direction order of the
    D3Q19 weights given here (rest, 6 faces, 12 edges; weights 1/3, 1/18,
    1/36).  Non-fluid entries are set to the rest weights as well; consumers
    ignore them.
    """
    nx, ny, nz = inst.shape
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=np.float64)
    rng = np.random.default_rng(seed)
    pert = rng.uniform(-1.0, 1.0, size=(19, nx * ny * nz))
    return w[:, None] * (1.0 + amp * pert)


def ib_ring_nodes(cx: float, cy: float, radius: float, z_centres, seed: int,
                  k_nominal: float, alpha: float, beta: float, ms: float,
                  pin_ends: bool = True):
    """Lagrangian wall nodes on a cylinder of the given radius: one ring per
    z in ``z_centres`` with round(2 pi R) nodes at unit arc spacing; area
    weight = arc length x ring spacing; stiffness k_nominal x U[0.5, 2]
    (seeded); the first and last ring pinned."""
    from .spec import IBNodes
    rng = np.random.default_rng(seed)
    n_th = max(8, int(round(2 * np.pi * radius)))
    th = 2 * np.pi * np.arange(n_th) / n_th
    z_centres = np.asarray(z_centres, dtype=np.float64)
    dz = float(z_centres[1] - z_centres[0]) if z_centres.size > 1 else 1.0
    X = np.empty((z_centres.size * n_th, 3))
    X[:, 0] = np.tile(cx + radius * np.cos(th), z_centres.size)
    X[:, 1] = np.tile(cy + radius * np.sin(th), z_centres.size)
    X[:, 2] = np.repeat(z_centres, n_th)
    ns = X.shape[0]
    dA = np.full(ns, 2 * np.pi * radius / n_th * dz)
    ks = k_nominal * rng.uniform(0.5, 2.0, ns)
    pinned = np.zeros(ns, np.uint8)
    if pin_ends:
        pinned[:n_th] = 1
        pinned[-n_th:] = 1
    return IBNodes(X0=X, dA=dA, ks=ks, pinned=pinned, alpha=alpha, beta=beta, ms=ms)


# penalty gains and wall parameters of the elastic-wall workloads (lattice
# units; the paper takes alpha, beta from earlier work without values)
IB_ALPHA, IB_BETA, IB_MS, IB_K = -2.0e-3, -0.5, 1.0, 0.01


# stretching and bending stiffness of the filament wall (lattice units, per
# unit width; explicit stability with m_s = 1 needs Eh < 1 and EI < 1/4)
FIL_EH, FIL_EI = 0.1, 0.02


def ib_tube(nx: int = 20, ny: int = 20, nz: int = 24, radius: float = 5.0,
            margin: float = 3.0, tau: float = 0.8, u_peak: float = 0.01,
            period: int = 400, seed: int = 0, filaments: bool = False) -> Instance:
    """Straight tube whose wall is a ring of Lagrangian nodes at ``radius``.

    Fluid fills r < radius + margin so the kernel support of every wall node
    lies in fluid; the 0D inlet (Womersley profile) and RCR outlet cover
    r < radius only, the jacket outside the membrane is closed at both ends.
    ``filaments``: every axial line of nodes (one per angle) is also an SGFD
    filament (ds = 1, Eh = FIL_EH, EI = FIL_EI), pinned at both end rings.
    """
    node = geometry.straight_tube(nx, ny, nz, radius + margin)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5, indexing="xy")
    outer = (X - nx / 2) ** 2 + (Y - ny / 2) ** 2 >= radius * radius
    node[0][outer] = 1
    node[nz - 1][outer] = 1
    inst = Instance(node=node, tau=tau, name=f"ib_tube_{nx}x{ny}x{nz}_R{radius:g}")
    omega = 2.0 * np.pi / period
    r = geometry.node_radius(nx, ny, inst.boundary_nodes(0))
    prof = profiles.womersley_coefficients(r, radius, omega, viscosity(tau), u_peak)
    inst.boundaries.append(Boundary(BC_VELOCITY, 2, +1, [omega], profile=prof))
    inst.boundaries.append(Boundary(BC_RCR, 2, -1, [0.05, 200.0, 1.0, 0.0]))
    inst.ib = ib_ring_nodes(nx / 2, ny / 2, radius, np.arange(1, nz - 1) + 0.5, seed,
                            IB_K, IB_ALPHA, IB_BETA, IB_MS)
    if filaments:
        n_rings = nz - 2
        n_th = inst.ib.n // n_rings
        inst.ib.filaments = [j + n_th * np.arange(n_rings) for j in range(n_th)]
        inst.ib.fil_par = np.tile([1.0, FIL_EH, FIL_EI], (n_th, 1))
        inst.name += "_filaments"
    return inst
