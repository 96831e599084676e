"""Plain data containers describing one lattice instance.

Layout conventions shared by every consumer:

* ``node`` is a ``uint8`` array of shape ``(nz, ny, nx)``; the flat cell
  index is ``x + nx*(y + ny*z)``.  Lattice node ``(x, y, z)`` sits at the
  physical position ``(x + 0.5, y + 0.5, z + 0.5)`` (lattice units,
  dx = dt = 1).
* node codes: ``0`` fluid (the domain Omega), ``1`` rigid wall (halfway
  bounce-back), ``2 + k`` a node of the 0D-coupled boundary ``k`` (part of
  the paper's boundary set dOmega_2, Section 2.1).
* boundary ``k`` has an inward unit normal ``sign * e_axis``: the fluid lies
  on that side of its node plane.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

NODE_FLUID = 0
NODE_WALL = 1
NODE_BOUNDARY0 = 2
MAX_BOUNDARIES = 8

# Boundary kinds (how the 0D side sets P* and v* of the non-equilibrium
# extrapolation, Section 2.2).
BC_VELOCITY = 0   # prescribed velocity profile u(x_b, t) (velocity-type coupling)
BC_RCR = 1        # three-element Windkessel outlet (pressure-type coupling)
BC_LV = 2         # left-ventricle elastance inlet with valve switching (hybrid)
BC_PRESSURE = 3   # constant gauge pressure (pressure-type coupling)


@dataclass
class Boundary:
    """One 0D-coupled boundary.

    ``params`` by kind:

    * BC_VELOCITY: ``[omega]``; ``profile`` is ``(n_nodes, 3)`` float64 with
      columns ``u_mean, c_re, c_im`` in raster order of the boundary's nodes;
      the prescribed normal velocity is ``u_mean + Re{(c_re + i c_im) e^{i omega t}}``.
    * BC_RCR: ``[R_p, C, R_d, P_w0(, order)]`` (characteristic impedance,
      compliance, peripheral resistance, initial chamber pressure; gauge
      units; optional marching order 1, 2 or 4).
    * BC_LV: ``[period_steps, P_la, N_S, P_v0(, order)]``; ``elastance`` is a
      ``(period_steps, 2)`` float64 table of ``E(t)`` and ``dE/dt`` at
      integer steps ``t mod period``.
    * BC_PRESSURE: ``[p_gauge]``.
    """
    kind: int
    axis: int
    sign: int
    params: List[float]
    profile: Optional[np.ndarray] = None
    elastance: Optional[np.ndarray] = None


@dataclass
class IBNodes:
    """Lagrangian wall nodes for the penalty immersed boundary (Section 2.3.2).

    ``X0`` reference positions ``(ns, 3)``; ``dA`` area weights; ``ks``
    spring stiffness per node; ``pinned`` 1 for nodes held at ``X0``;
    ``alpha``/``beta`` the (negative) penalty gains; ``ms`` wall mass per area.

    Optional filaments (the SGFD solid of Section 2.3.2): ``filaments`` a list
    of node-index arrays in arc-length order, ``fil_par`` ``(n_fil, 3)`` with
    ``(ds, Eh, EI)`` per filament.  Their interior nodes add the tension and
    bending forces to the spring; their end nodes must be pinned.
    """
    X0: np.ndarray
    dA: np.ndarray
    ks: np.ndarray
    pinned: np.ndarray
    alpha: float
    beta: float
    ms: float
    filaments: Optional[List[np.ndarray]] = None
    fil_par: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.X0.shape[0])


@dataclass
class Instance:
    """A lattice, its relaxation time, 0D boundaries and optional IB wall.

    ``q_scale``: 1 feeds the 0D models the area-mean velocity Q/A of the
    boundary's first fluid layer, 0 feeds the literal flow Q.
    """
    node: np.ndarray
    tau: float
    boundaries: List[Boundary] = field(default_factory=list)
    ib: Optional[IBNodes] = None
    q_scale: int = 1
    name: str = ""

    @property
    def shape(self):
        nz, ny, nx = self.node.shape
        return nx, ny, nz

    @property
    def n_fluid(self) -> int:
        return int((self.node == NODE_FLUID).sum())

    def boundary_nodes(self, k: int) -> np.ndarray:
        """Flat indices (raster order) of the nodes of boundary ``k``."""
        return np.flatnonzero(self.node.reshape(-1) == NODE_BOUNDARY0 + k)
