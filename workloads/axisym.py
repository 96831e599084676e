"""Inputs of the axisymmetric (D2Q9, pseudo-Cartesian (x, r)) workloads.

A node array has shape ``(nr, nx)``; node ``(x, j)`` sits at
``r = j + 1/2`` (the symmetry axis lies below row 0) and codes are those of
the 3D lattices: 0 fluid, 1 rigid wall, 2 + k node of 0D boundary k.
0D boundaries are node columns at ``x = 0`` (inward normal +e_x, sign +1)
or ``x = nx - 1`` (sign -1), axis 0; a velocity profile lists one entry per
boundary node in increasing r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import configs, profiles
from .spec import BC_LV, BC_RCR, BC_VELOCITY, Boundary


@dataclass
class AxiInstance:
    node: np.ndarray
    tau: float
    boundaries: List[Boundary] = field(default_factory=list)
    q_scale: int = 1
    name: str = ""

    @property
    def shape(self):
        nr, nx = self.node.shape
        return nx, nr


def pipe(nr: int, nx: int, radius: float) -> np.ndarray:
    """Straight pipe of the given wall radius with 0D boundary columns
    (codes 2 at x = 0 and 3 at x = nx - 1) over the lumen."""
    r = np.arange(nr) + 0.5
    node = np.where(r[:, None] < radius, 0, 1).astype(np.uint8) * np.ones((1, nx), np.uint8)
    node[:, 0] = np.where(r < radius, 2, 1)
    node[:, -1] = np.where(r < radius, 3, 1)
    return node


def stenosis(nr: int, nx: int, r0: float, depth: float, width: float):
    """Pipe of radius r0 narrowed by a Gaussian of the given depth and width
    around x = nx/2; returns (node, R(x))."""
    x = np.arange(nx) + 0.5
    r = np.arange(nr) + 0.5
    R = r0 - depth * np.exp(-((x - nx / 2) / width) ** 2)
    node = np.where(r[:, None] < R[None, :], 0, 1).astype(np.uint8)
    node[:, 0] = np.where(r < r0, 2, 1)
    node[:, -1] = np.where(r < r0, 3, 1)
    return node, R


def womersley_tube(nr: int = 10, nx: int = 48, radius: float = 8.0, tau: float = 0.8,
                   u_peak: float = 0.02, period: int = 400,
                   rcr=(0.05, 200.0, 1.0, 0.0)) -> AxiInstance:
    """Rigid pipe with a Womersley velocity inlet and an RCR outlet."""
    node = pipe(nr, nx, radius)
    inst = AxiInstance(node=node, tau=tau, name=f"axi_womersley_{nx}x{nr}_R{radius:g}")
    omega = 2 * math.pi / period
    r = np.arange(int((node[:, 0] == 2).sum())) + 0.5
    prof = profiles.womersley_coefficients(r, radius, omega, configs.viscosity(tau), u_peak)
    inst.boundaries.append(Boundary(BC_VELOCITY, 0, +1, [omega], profile=prof))
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, list(rcr)))
    return inst


def lv_tube(nr: int = 8, nx: int = 40, radius: float = 6.0, tau: float = 0.8,
            period: int = 600) -> AxiInstance:
    """Rigid pipe with the hybrid LV inlet and an RCR outlet (the 3D LV
    tube's 0D parameters: elastance scale x 4000/period, R_p = 0.02,
    C = 1200, R_d = 1)."""
    node = pipe(nr, nx, radius)
    inst = AxiInstance(node=node, tau=tau, name=f"axi_lv_{nx}x{nr}_R{radius:g}_T{period}")
    inst.boundaries.append(configs.lv_boundary(period=period, kappa=configs.LV_KAPPA * 4000.0 / period,
                                               axis=0, sign=+1))
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, [0.02, 1200.0, 1.0, 0.0]))
    return inst
