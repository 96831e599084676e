"""Pins of the Womersley inlet coefficients (workloads.profiles.womersley_coefficients).

Both the oracle and the CUDA path consume these per-node coefficients, so a
mistake in them would be shared by both sides of every parity test; they are
pinned here against what the tube problem itself fixes (the reading of the
workload's Womersley inlet: zero-mean oscillating pressure gradient, velocity
u(r, t) = Re{c(r) e^{i w t}}):

* c solves the oscillatory tube equation  i w c = G + nu (c'' + c'/r)  for one
  constant G: nu (c'' + c'/r) - i w c, by central finite differences of the
  returned profile, is the same at every radius (a wrong sign of i^{3/2}, the
  conjugate time convention or a wrong Womersley number R sqrt(w/nu) breaks it);
* no slip, c(R) = 0, and regularity on the axis, c'(0) = 0;
* the amplitude: max_r |c| = u_peak over the radii given;
* the small-Womersley-number limit is the Poiseuille parabola 1 - r^2/R^2;
* J0 of the complex arguments used agrees with the power series of
  Abramowitz & Stegun 9.1.10, summed here independently of scipy.
"""
import math

import numpy as np
import pytest

from workloads import profiles


def _c(r, R, w, nu, u):
    out = profiles.womersley_coefficients(np.asarray(r, dtype=np.float64), R, w, nu, u)
    assert np.all(out[:, 0] == 0.0)            # zero-mean profile
    return out[:, 1] + 1j * out[:, 2]


@pytest.mark.parametrize("R,period,tau", [(8.0, 1000, 0.8), (5.0, 400, 0.8), (20.0, 4000, 0.55), (6.0, 200, 1.2)])
def test_tube_equation(R, period, tau):
    w = 2 * np.pi / period
    nu = (tau - 0.5) / 3
    u = 0.02
    # the profile scales to max |c| = u over the radii passed: pass the same set each time
    r = np.linspace(0.1 * R, 0.95 * R, 18)
    h = 1e-3 * R
    grid = np.concatenate([r - h, r, r + h, np.linspace(0, R, 2001)])
    c = _c(grid, R, w, nu, u)
    cm, c0, cp = c[:18], c[18:36], c[36:54]
    lap = (cp - 2 * c0 + cm) / h ** 2 + (cp - cm) / (2 * h) / r
    L = nu * lap - 1j * w * c0
    scale = w * np.abs(c).max()
    assert np.abs(L - L.mean()).max() < 1e-5 * scale
    assert np.abs(L.mean()) > 0.1 * scale      # a real driving gradient


def test_no_slip_regular_axis_and_amplitude():
    R, w, nu, u = 8.0, 2 * np.pi / 1000, 0.1, 0.02
    r = np.concatenate([[0.0, 1e-3, R], np.linspace(0, R, 4001)])
    c = _c(r, R, w, nu, u)
    assert abs(c[2]) < 1e-15
    assert abs(c[1] - c[0]) < 1e-6 * abs(c[0])             # c'(0) = 0: O(h^2) change
    assert np.abs(c).max() == pytest.approx(u, rel=1e-14)


def test_small_womersley_number_is_poiseuille():
    R, nu, u = 10.0, 0.1, 0.02
    alpha = 0.05
    w = nu * (alpha / R) ** 2
    r = np.linspace(0, R, 201)
    c = _c(r, R, w, nu, u)
    assert np.abs(np.abs(c) / np.abs(c[0]) - (1 - (r / R) ** 2)).max() < 1e-3
    assert np.abs(c).argmax() == 0                        # largest on the axis


def _j0_series(z):
    """J0(z) = sum_k (-z^2/4)^k / (k!)^2 (Abramowitz & Stegun 9.1.10)."""
    t = -0.25 * z * z
    s, term = 0j, 1 + 0j
    for k in range(200):
        if k:
            term *= t / (k * k)
        s += term
        if abs(term) < 1e-18 * max(abs(s), 1.0):
            break
    return s


@pytest.mark.parametrize("alpha", [0.5, 2.0, 4.0, 8.0])
def test_shape_against_series(alpha):
    R = 8.0
    nu = 0.1
    w = nu * (alpha / R) ** 2
    r = np.linspace(0, R, 33)
    c = _c(r, R, w, nu, 1.0)
    i32 = complex(math.cos(0.75 * math.pi), math.sin(0.75 * math.pi))
    shape = np.array([1 - _j0_series(i32 * alpha * x / R) / _j0_series(i32 * alpha) for x in r])
    ref = shape / np.abs(shape).max()
    assert np.abs(c - ref).max() < 1e-12
