"""Parameter-sweep batches of rigid tubes (the batching and warm-start workloads).

``tube_batch``: instances of uneven size -- radius uniform in [6, 20], length
uniform in [128, 512], square box of side ceil(2R + 4) -- each with an LV
elastance inlet (E_max uniform in [1.5, 3.0], E_min = 0.06, period uniform in
[2000, 6000] steps, all times the lattice elastance scale) and an RCR outlet
whose resistances are log-uniform within +-50 % of the rigid-tube workload's
(R_p = 0.05, R_d = 1.0).  The compliance is log-uniform within +-50 % of
C = 1.5 T / R_d, so that the Windkessel time constant R_d C is 1.5 beats, as
in a physiological arterial tree; with the rigid-tube workload's C = 200
(R_d C = 0.2 of its 1000-step beat) the chamber would empty between beats
of an LV inlet.

``lv_sweep``: the warm-start workload on one geometry -- the same six 0D
parameters (R_p, C, R_d, E_max, E_min, period) drawn for many copies of one
small tube.

``lv_geometry_sweep``: the warm-start workload over the batching workload's
geometries -- radius uniform in [6, 20] and length uniform in [128, 512]
drawn per instance together with the six 0D parameters.
"""
from __future__ import annotations

import math

import numpy as np

from . import configs, geometry
from .spec import BC_RCR, Boundary, Instance

PARAM_NAMES = ("R_p", "C", "R_d", "E_max", "E_min", "period")


def draw_params(rng: np.random.Generator, n: int, e_min_range=(0.06, 0.06),
                period_step: int = 1, period_range=(2000, 6000)) -> np.ndarray:
    """(n, 6) array of (R_p, C, R_d, E_max, E_min, period)."""
    lo, hi = math.log(0.5), math.log(1.5)
    Rp = 0.05 * np.exp(rng.uniform(lo, hi, n))
    Rd = 1.0 * np.exp(rng.uniform(lo, hi, n))
    T = rng.uniform(period_range[0], period_range[1], n)
    T = np.round(T / period_step) * period_step
    C = 1.5 * T / 1.0 * np.exp(rng.uniform(lo, hi, n))
    Emax = rng.uniform(1.5, 3.0, n)
    Emin = rng.uniform(e_min_range[0], e_min_range[1], n)
    return np.stack([Rp, C, Rd, Emax, Emin, T], axis=1)


def lv_tube_instance(params, radius: float, length: int, tau: float = 0.8,
                     kappa: float = configs.LV_KAPPA) -> Instance:
    """Rigid tube of the given radius and length with an LV inlet and an RCR
    outlet set from one row of :func:`draw_params` (``kappa``: the lattice
    elastance scale)."""
    Rp, C, Rd, Emax, Emin, T = (float(v) for v in params)
    n_xy = int(math.ceil(2 * radius + 4))
    node = geometry.straight_tube(n_xy, n_xy, int(length), radius)
    inst = Instance(node=node, tau=tau, name=f"lv_tube_R{radius:.2f}_L{length}_T{int(T)}")
    inst.boundaries.append(configs.lv_boundary(period=int(T), e_max=Emax, e_min=Emin, kappa=kappa))
    inst.boundaries.append(Boundary(BC_RCR, 2, -1, [Rp, C, Rd, 0.0]))
    return inst


def tube_batch(n: int = 256, seed: int = 0):
    """Returns (instances, params) for the uneven-size batching workload."""
    rng = np.random.default_rng(seed)
    params = draw_params(rng, n)
    R = rng.uniform(6.0, 20.0, n)
    L = rng.integers(128, 513, n)
    return [lv_tube_instance(params[q], R[q], int(L[q])) for q in range(n)], params


def lv_sweep(n: int, seed: int, radius: float = 6.0, length: int = 128, period_step: int = 100,
             period_range=(2000, 6000), kappa: float = configs.LV_KAPPA):
    """Returns (instances, params) for the warm-start study: one tube
    geometry, six 0D parameters drawn per instance (periods on a grid of
    ``period_step`` steps so that a batch can be read at every instance's
    cycle phase 0 after a whole number of chunks)."""
    rng = np.random.default_rng(seed)
    params = draw_params(rng, n, e_min_range=(0.05, 0.07), period_step=period_step,
                         period_range=period_range)
    return [lv_tube_instance(params[q], radius, length, kappa=kappa) for q in range(n)], params


def lv_geometry_sweep(n: int, seed: int, period_step: int = 100, period_range=(2000, 6000),
                      radius_range=(6.0, 20.0), length_range=(128, 512), kappa: float = configs.LV_KAPPA):
    """Returns (instances, params, geometry) for the warm-start study over the
    batching workload's geometries: ``geometry[q] = (R, L)``; six 0D
    parameters drawn per instance as in :func:`lv_sweep`."""
    rng = np.random.default_rng(seed)
    params = draw_params(rng, n, e_min_range=(0.05, 0.07), period_step=period_step, period_range=period_range)
    R = rng.uniform(radius_range[0], radius_range[1], n)
    L = rng.integers(length_range[0], length_range[1] + 1, n)
    geom = np.stack([R, L.astype(np.float64)], axis=1)
    return [lv_tube_instance(params[q], R[q], int(L[q]), kappa=kappa) for q in range(n)], params, geom
