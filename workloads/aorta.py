"""Synthetic aorta-like vessel (the full-size elastic-wall workload).

128 x 128 x 1024 lattice.  The centreline is a natural cubic spline through
five control points at z = 0, 256, 512, 768, 1024 with seeded lateral
offsets in [-16, 16]; the radius tapers linearly from 40 to 24.  The vessel
wall is a membrane of Lagrangian nodes on r = R(z) (about 2e5 nodes at unit
area spacing, linear springs with stiffness drawn uniformly in
[0.5, 2] x nominal (:data:`AORTA_K`), end rings pinned); the fluid fills r < R(z) + 3 so that
the support of every wall node lies in fluid, and rigid bounce-back walls
bound it beyond.  Two rigid side branches of radius 10 leave along +x and
-x at seeded heights z in [300, 700] and end on the x faces.

0D boundaries: LV elastance inlet at z = 0 (E_max = 2.0, E_min = 0.06 in the
lattice scaling of :data:`workloads.configs.LV_KAPPA`, period 4000 steps),
RCR Windkessel at z = nz - 1 and on both branch ends.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import CubicSpline

from . import configs
from .spec import BC_RCR, NODE_BOUNDARY0, NODE_FLUID, NODE_WALL, Boundary, Instance

NX, NY, NZ = 128, 128, 1024
R_IN, R_OUT, R_BRANCH, JACKET = 40.0, 24.0, 10.0, 3.0
# Nominal tether stiffness of the membrane nodes.  At the tube workloads'
# 0.01 the nodes on the rim of the branch holes, dragged by the outflow into
# the branches, creep outwards beat after beat (peak displacement 0.71, 0.89,
# 0.98 ... 1.25 cells) until one leaves its 6^3 support box in the seventh
# beat; at 0.04 the peak displacement levels off near 0.41 cells over ten
# beats (the workload's 4e4 steps) and the median stays below 0.004 cells.
AORTA_K = 0.04


def centreline(seed: int, nz: int = NZ, cx: float = NX / 2, cy: float = NY / 2, amp: float = 16.0):
    """(x_c(z), y_c(z)) at the cell-centre heights z + 0.5."""
    rng = np.random.default_rng(seed)
    zc = np.linspace(0.0, float(nz), 5)
    offs = rng.uniform(-amp, amp, size=(5, 2))
    z = np.arange(nz) + 0.5
    sx = CubicSpline(zc, offs[:, 0], bc_type="natural")(z)
    sy = CubicSpline(zc, offs[:, 1], bc_type="natural")(z)
    return cx + np.clip(sx, -amp, amp), cy + np.clip(sy, -amp, amp)


def radius(nz: int = NZ, r_in: float = R_IN, r_out: float = R_OUT):
    z = np.arange(nz) + 0.5
    return r_in + (r_out - r_in) * z / nz


def build(seed: int = 0, nx: int = NX, ny: int = NY, nz: int = NZ, period: int = 4000,
          with_ib: bool = True) -> Instance:
    xc, yc = centreline(seed, nz)
    R = radius(nz)
    rng = np.random.default_rng(seed + 1000)
    zb = rng.uniform(300.0 * nz / NZ, 700.0 * nz / NZ, size=2)
    X = np.arange(nx) + 0.5
    Y = np.arange(ny) + 0.5
    XX, YY = np.meshgrid(X, Y, indexing="xy")
    node = np.full((nz, ny, nx), NODE_WALL, dtype=np.uint8)
    for z in range(1, nz - 1):
        d2 = (XX - xc[z]) ** 2 + (YY - yc[z]) ** 2
        node[z][d2 < (R[z] + JACKET) ** 2] = NODE_FLUID
    # branches: +x (k = 0) and -x (k = 1), axis along x at (y_c(z_b), z_b)
    branch_axes = []
    for k, sgn in enumerate((+1, -1)):
        zi = int(zb[k])
        ya, za = yc[zi], zb[k]
        branch_axes.append((sgn, ya, za, xc[zi]))
        zs = np.arange(max(1, int(za - R_BRANCH - 2)), min(nz - 1, int(za + R_BRANCH + 3)))
        for z in zs:
            d2 = (YY - ya) ** 2 + (z + 0.5 - za) ** 2
            inside = d2 < R_BRANCH ** 2
            side = (XX - xc[zi]) * sgn > 0
            node[z][inside & side] = NODE_FLUID
    # 0D boundary nodes
    d2 = (XX - xc[0]) ** 2 + (YY - yc[0]) ** 2
    node[0][d2 < R[0] ** 2] = NODE_BOUNDARY0 + 0                  # LV inlet
    d2 = (XX - xc[nz - 1]) ** 2 + (YY - yc[nz - 1]) ** 2
    node[nz - 1][d2 < R[nz - 1] ** 2] = NODE_BOUNDARY0 + 1        # aortic outlet
    for k, (sgn, ya, za, _) in enumerate(branch_axes):
        xf = nx - 1 if sgn > 0 else 0
        Z, Yv = np.meshgrid(np.arange(nz) + 0.5, Y, indexing="ij")
        face = (Yv - ya) ** 2 + (Z - za) ** 2 < R_BRANCH ** 2
        node[:, :, xf][face] = NODE_BOUNDARY0 + 2 + k
    inst = Instance(node=node, tau=0.8, name=f"aorta_{nx}x{ny}x{nz}_seed{seed}")
    inst.boundaries.append(configs.lv_boundary(period=period))
    inst.boundaries.append(Boundary(BC_RCR, 2, -1, [0.01, 10000.0, 0.3, 0.0]))
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, [0.05, 2000.0, 1.0, 0.0]))
    inst.boundaries.append(Boundary(BC_RCR, 0, +1, [0.05, 2000.0, 1.0, 0.0]))
    if with_ib:
        inst.ib = wall_nodes(xc, yc, R, branch_axes, seed)
    return inst


def wall_nodes(xc, yc, R, branch_axes, seed: int):
    """Membrane nodes: one ring per interior cell height, round(2 pi R) nodes
    per ring, minus a hole of radius R_branch + 2 around each branch axis."""
    from .spec import IBNodes
    nz = R.size
    rng = np.random.default_rng(seed + 2000)
    pts, dA, ring = [], [], []
    for z in range(1, nz - 1):
        n_th = int(round(2 * np.pi * R[z]))
        th = 2 * np.pi * np.arange(n_th) / n_th
        x = xc[z] + R[z] * np.cos(th)
        y = yc[z] + R[z] * np.sin(th)
        keep = np.ones(n_th, bool)
        for sgn, ya, za, _ in branch_axes:
            near = ((y - ya) ** 2 + (z + 0.5 - za) ** 2 < (R_BRANCH + 2.0) ** 2) & ((x - xc[z]) * sgn > 0)
            keep &= ~near
        pts.append(np.stack([x[keep], y[keep], np.full(keep.sum(), z + 0.5)], axis=1))
        dA.append(np.full(keep.sum(), 2 * np.pi * R[z] / n_th))
        ring.append(np.full(keep.sum(), z))
    X0 = np.concatenate(pts)
    dA = np.concatenate(dA)
    ring = np.concatenate(ring)
    pinned = ((ring == 1) | (ring == nz - 2)).astype(np.uint8)
    ks = AORTA_K * rng.uniform(0.5, 2.0, X0.shape[0])
    return IBNodes(X0=X0, dA=dA, ks=ks, pinned=pinned, alpha=configs.IB_ALPHA,
                   beta=configs.IB_BETA, ms=configs.IB_MS)
