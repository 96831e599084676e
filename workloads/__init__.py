"""Seeded synthetic inputs for the 0D-3D lattice Boltzmann hot path.

This package builds problem *inputs* only: node-type lattices (fluid, rigid
wall, 0D boundary nodes), prescribed inlet velocity profiles, the ventricular
elastance curve sampled per time step, Lagrangian wall-node sets and the 0D
parameters.  It holds none of the method's arithmetic (no equilibrium,
collision, streaming, non-equilibrium extrapolation, ODE step or immersed
boundary kernel), so the CPU oracle and the CUDA path can both consume it
without sharing any of the computation they are compared on.

Algorithm 1 of the paper lists the elastance curve C_v(t) and its time
derivative as *inputs* of the solver (Section 2.1.2 allows a look-up table);
they are therefore generated here, per integer time step.
"""
from .spec import (  # noqa: F401
    BC_VELOCITY, BC_RCR, BC_LV, BC_PRESSURE,
    NODE_FLUID, NODE_WALL, NODE_BOUNDARY0,
    Boundary, IBNodes, Instance,
)
from . import geometry, configs  # noqa: F401
