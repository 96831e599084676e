"""Node-type lattices for tubes, boxes and the synthetic aorta.

Pure geometry: which lattice node is fluid, rigid wall or a 0D boundary
node.  Cell centres sit at ``index + 0.5``.
"""
from __future__ import annotations

import numpy as np

from .spec import NODE_BOUNDARY0, NODE_FLUID, NODE_WALL


def _centres(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) + 0.5


def straight_tube(nx: int, ny: int, nz: int, radius: float,
                  cx: float | None = None, cy: float | None = None,
                  inlet: bool = True, outlet: bool = True) -> np.ndarray:
    """Rigid straight tube along z.

    Fluid where the cell centre is closer than ``radius`` to the axis, for
    ``1 <= z <= nz-2``; the planes ``z = 0`` and ``z = nz-1`` hold the nodes
    of boundary 0 (inlet) and boundary 1 (outlet) inside the radius (or
    wall when the flag is off); everything else is wall.
    """
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    X, Y = np.meshgrid(_centres(nx), _centres(ny), indexing="xy")
    inside = (X - cx) ** 2 + (Y - cy) ** 2 < radius * radius
    node = np.full((nz, ny, nx), NODE_WALL, dtype=np.uint8)
    node[1:nz - 1][:, inside] = NODE_FLUID
    if inlet:
        node[0][inside] = NODE_BOUNDARY0 + 0
    if outlet:
        node[nz - 1][inside] = NODE_BOUNDARY0 + (1 if inlet else 0)
    return node


def closed_box(nx: int, ny: int, nz: int) -> np.ndarray:
    """Fluid interior surrounded by a one-cell rigid wall shell."""
    node = np.full((nz, ny, nx), NODE_WALL, dtype=np.uint8)
    node[1:-1, 1:-1, 1:-1] = NODE_FLUID
    return node


def plates_channel(nx: int, ny: int, nz: int) -> np.ndarray:
    """Fluid between two wall planes ``y = 0`` and ``y = ny-1``; all other
    directions are meant to be periodic (oracle-only pins)."""
    node = np.full((nz, ny, nx), NODE_FLUID, dtype=np.uint8)
    node[:, 0, :] = NODE_WALL
    node[:, ny - 1, :] = NODE_WALL
    return node


def periodic_tube(nx: int, ny: int, nz: int, radius: float) -> np.ndarray:
    """Tube along z with no end planes (z meant to be periodic)."""
    X, Y = np.meshgrid(_centres(nx), _centres(ny), indexing="xy")
    inside = (X - nx / 2.0) ** 2 + (Y - ny / 2.0) ** 2 < radius * radius
    node = np.full((nz, ny, nx), NODE_WALL, dtype=np.uint8)
    node[:, inside] = NODE_FLUID
    return node


def node_radius(nx: int, ny: int, flat_idx: np.ndarray,
                cx: float | None = None, cy: float | None = None) -> np.ndarray:
    """Distance of cell centres (given by flat index) from a z-parallel axis."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    x = flat_idx % nx
    y = (flat_idx // nx) % ny
    return np.hypot(x + 0.5 - cx, y + 0.5 - cy)
