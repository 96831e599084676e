"""Prescribed boundary data: inlet velocity profiles and elastance curves.

Both are inputs of the solver (Algorithm 1 lists C_v(t) and dC_v/dt among
its inputs; the inlet profile of the rigid-tube workload is a prescribed
Dirichlet velocity).
"""
from __future__ import annotations

import numpy as np
from scipy import special


def womersley_coefficients(r: np.ndarray, radius: float, omega: float,
                           nu: float, u_peak: float) -> np.ndarray:
    """Complex amplitude ``c(r)`` of the oscillatory Womersley tube profile.

    u(r, t) = Re{c(r) e^{i omega t}} with
    c(r) = A [1 - J0(i^{3/2} a r / R) / J0(i^{3/2} a)],  a = R sqrt(omega/nu)
    (zero-mean pressure-gradient solution).  ``A`` is real and chosen so that
    max_r |c(r)| over the given radii equals ``u_peak``; since
    max_t Re{c e^{i w t}} = |c|, the largest prescribed velocity is u_peak.
    Returns an ``(n, 3)`` array ``[u_mean=0, Re c, Im c]``.
    """
    a = radius * np.sqrt(omega / nu)
    i32 = np.exp(1j * 0.75 * np.pi)  # i^{3/2}
    shape = 1.0 - special.jv(0, i32 * a * r / radius) / special.jv(0, i32 * a)
    amp = u_peak / np.max(np.abs(shape))
    c = amp * shape
    out = np.zeros((r.shape[0], 3), dtype=np.float64)
    out[:, 1] = c.real
    out[:, 2] = c.imag
    return out


def plug_profile(n: int, u: float) -> np.ndarray:
    """Steady uniform normal velocity ``u`` on ``n`` nodes."""
    out = np.zeros((n, 3), dtype=np.float64)
    out[:, 0] = u
    return out


# Double-Hill elastance shape (Stergiopulos, Meister & Westerhof 1996),
# commonly quoted parameters.
HILL_A1, HILL_A2, HILL_N1, HILL_N2 = 0.303, 0.508, 1.32, 21.9


def _hill_shape(tau_rel: np.ndarray, a1: float, a2: float, n1: float, n2: float):
    """Unnormalised double-Hill g(t) and dg/d(tau_rel) for tau_rel = t / T."""
    r1 = (tau_rel / a1) ** n1
    r2 = (tau_rel / a2) ** n2
    g1 = r1 / (1.0 + r1)
    g2 = 1.0 / (1.0 + r2)
    with np.errstate(divide="ignore", invalid="ignore"):
        dr1 = np.where(tau_rel > 0, n1 * r1 / tau_rel, 0.0)
        dr2 = np.where(tau_rel > 0, n2 * r2 / tau_rel, 0.0)
    dg1 = dr1 / (1.0 + r1) ** 2
    dg2 = -dr2 / (1.0 + r2) ** 2
    return g1 * g2, dg1 * g2 + g1 * dg2


def elastance_table(period: int, e_max: float, e_min: float,
                    a1: float = HILL_A1, a2: float = HILL_A2,
                    n1: float = HILL_N1, n2: float = HILL_N2,
                    n_norm: int = 200001) -> np.ndarray:
    """``(period, 2)`` table of E(t) and dE/dt at integer steps t.

    E(t) = (E_max - E_min) * g(t mod T) / max g + E_min, with the normalising
    maximum found by dense FP64 sampling over one period.  dE/dt is the
    analytic derivative of the same curve (per step).
    """
    dense = np.linspace(0.0, 1.0, n_norm)
    gmax = float(_hill_shape(dense, a1, a2, n1, n2)[0].max())
    t = np.arange(period, dtype=np.float64) / period
    g, dg = _hill_shape(t, a1, a2, n1, n2)
    tab = np.empty((period, 2), dtype=np.float64)
    tab[:, 0] = (e_max - e_min) * g / gmax + e_min
    tab[:, 1] = (e_max - e_min) * dg / gmax / period
    return tab
