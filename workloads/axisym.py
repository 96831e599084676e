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
from .spec import BC_RCR, BC_VELOCITY, Boundary


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


# The straight-aorta convergence workload (Section 3.1.3's axisymmetric
# aorta, 25 diameters long, LV inlet, Womersley number 16) under diffusive
# scaling.  Lattice parameters are fixed at the reference resolution of
# E5_REF_ND = 20 nodes per diameter and a 100-step beat (tau = 0.574,
# elastance scale 0.013, Windkessel R_p = 0.05, C = 150, R_d = 1: one valve
# opening per beat, time constant 1.5 beats) and carried to other
# resolutions by the unit scales: velocity dt/dx, pressure (dt/dx)^2,
# resistance dt/dx, compliance dx/dt^2, elastance dt^2/dx.  The Reynolds
# number stays about 40 (the coarsest grid bounds the lattice Mach number).
E5_REF_ND, E5_REF_T = 20, 100
E5_KAPPA, E5_RCR = 0.013, (0.05, 150.0, 1.0)
E5_WOMERSLEY = 16.0


def e5_period(n_d: int) -> int:
    """Beat length in steps at n_d nodes per diameter (diffusive scaling,
    rounded to a multiple of 50 steps so that 50 phases are sampled)."""
    return max(50, int(round(E5_REF_T * (n_d / E5_REF_ND) ** 2 / 50.0)) * 50)


def straight_aorta(n_d: int, length_d: float = 25.0) -> AxiInstance:
    """The convergence workload at n_d nodes per diameter."""
    T = e5_period(n_d)
    radius = n_d / 2.0
    nr = int(math.ceil(radius))
    nx = int(round(length_d * n_d)) + 2
    node = pipe(nr, nx, radius)
    dx, dt = 1.0 / n_d, 1.0 / T
    dxr, dtr = 1.0 / E5_REF_ND, 1.0 / E5_REF_T
    nu_star = 2 * math.pi * 0.25 / E5_WOMERSLEY ** 2      # D = 1, beat = 1
    tau = 0.5 + 3.0 * nu_star * dt / dx ** 2
    s_u = (dt / dx) / (dtr / dxr)
    s_c = (dx / dt ** 2) / (dxr / dtr ** 2)
    s_e = (dt ** 2 / dx) / (dtr ** 2 / dxr)
    inst = AxiInstance(node=node, tau=tau, name=f"axi_aorta_D{n_d}_T{T}")
    lv = configs.lv_boundary(period=T, kappa=E5_KAPPA * s_e, p_la=configs.LV_P_LA * s_u * s_u, axis=0, sign=+1)
    inst.boundaries.append(lv)
    Rp, C, Rd = E5_RCR
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, [Rp * s_u, C * s_c, Rd * s_u, 0.0]))
    return inst


# The converging variant of the study: a straight tube of 4 diameters with a
# Womersley velocity inlet (Womersley number 4, the largest the rigid lattice
# resolves near its incompressible limit at 20 nodes per diameter: the
# acoustic transit of the tube is 0.12 beat there and shrinks under
# diffusive scaling) and an RCR outlet with a 1.5-beat time constant.
# Reference at 20 nodes per diameter: 1200-step beat (tau = 0.598), peak
# inlet velocity 0.02, R_p = 0.05, R_d = 1, C = 1800.
CONV_REF_T, CONV_U, CONV_RCR, CONV_WOMERSLEY, CONV_LENGTH_D = 1200, 0.02, (0.05, 1800.0, 1.0), 4.0, 4.0


def conv_period(n_d: int) -> int:
    """Beat in steps (diffusive scaling; a multiple of 40 for 40 phases)."""
    return int(round(CONV_REF_T * (n_d / E5_REF_ND) ** 2 / 40.0)) * 40


def convergence_tube(n_d: int) -> AxiInstance:
    """The converging study's tube at n_d nodes per diameter."""
    T = conv_period(n_d)
    radius = n_d / 2.0
    nr = int(math.ceil(radius))
    nx = int(round(CONV_LENGTH_D * n_d)) + 2
    node = pipe(nr, nx, radius)
    dx, dt = 1.0 / n_d, 1.0 / T
    dxr, dtr = 1.0 / E5_REF_ND, 1.0 / CONV_REF_T
    nu_star = 2 * math.pi * 0.25 / CONV_WOMERSLEY ** 2
    nu = nu_star * dt / dx ** 2
    s_u = (dt / dx) / (dtr / dxr)
    s_c = (dx / dt ** 2) / (dxr / dtr ** 2)
    inst = AxiInstance(node=node, tau=0.5 + 3.0 * nu, name=f"axi_conv_D{n_d}_T{T}")
    omega = 2 * math.pi / T
    r = np.arange(int((node[:, 0] == 2).sum())) + 0.5
    prof = profiles.womersley_coefficients(r, radius, omega, nu, CONV_U * s_u)
    inst.boundaries.append(Boundary(BC_VELOCITY, 0, +1, [omega], profile=prof))
    Rp, C, Rd = CONV_RCR
    inst.boundaries.append(Boundary(BC_RCR, 0, -1, [Rp * s_u, C * s_c, Rd * s_u, 0.0]))
    return inst
