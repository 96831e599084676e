"""Pins of the oracle's periodic-state criterion (oracle/periodic.py).

The criterion is not in the paper (which reads its results once the beats
repeat); its reading is fixed in the oracle's docstring.  The pins are closed
forms of waveform records built here, each chosen so that a plausible slip
in the definition fails one of them:

* an exactly periodic record gives 0;
* a record that grows by a factor 1 + eps per beat gives eps exactly (the
  previous beat is the denominator: normalising by the last beat would give
  eps / (1 + eps));
* a sine delayed by d steps from beat to beat gives 2 sin(pi d / T);
* the worst boundary and waveform decides; the chamber-state and valve
  columns do not count;
* only the last two beats count;
* fewer than 2 T rows give -1.
"""
import numpy as np
import pytest

import oracle


def _record(T, beats, nbc, fn):
    """rows [t, 4 values per boundary]; fn(t, k, col) fills value col of boundary k."""
    n = T * beats
    t = np.arange(n, dtype=np.float64)
    w = np.zeros((n, 1 + 4 * nbc))
    w[:, 0] = t
    for k in range(nbc):
        for col in range(4):
            w[:, 1 + 4 * k + col] = fn(t, k, col)
    return w


def test_periodic_record_gives_zero():
    T = 400
    w = _record(T, 4, 2, lambda t, k, col: np.sin(2 * np.pi * t / T + k + col) + 0.3 * np.cos(6 * np.pi * t / T))
    assert oracle.cycle_change(w, T) < 1e-13       # rounding of sin at t and t - T only


@pytest.mark.parametrize("eps", [1e-3, 0.02, 0.25])
def test_geometric_growth_gives_eps(eps):
    T = 360
    w = _record(T, 5, 1, lambda t, k, col: (1 + eps) ** np.floor(t / T) * np.sin(2 * np.pi * t / T + 0.1))
    assert oracle.cycle_change(w, T) == pytest.approx(eps, rel=1e-12)


@pytest.mark.parametrize("d", [2, 10, 40])
def test_delayed_sine(d):
    T = 1000
    # the beat c (t in [cT, (c+1)T)) is sin(omega (t - c d)): a delay of d steps per beat
    w = _record(T, 3, 1, lambda t, k, col: np.sin(2 * np.pi * (t - np.floor(t / T) * d) / T))
    assert oracle.cycle_change(w, T) == pytest.approx(2 * np.sin(np.pi * d / T), rel=1e-12)


def test_worst_channel_decides_and_state_columns_ignored():
    T = 200
    grow = {(0, 0): 0.01, (1, 1): 0.03, (0, 2): 0.5, (1, 3): 0.9}   # (boundary, column): growth per beat

    def fn(t, k, col):
        g = grow.get((k, col), 0.0)
        return (1 + g) ** np.floor(t / T) * (1.0 + 0.5 * np.sin(2 * np.pi * t / T))

    w = _record(T, 3, 2, fn)
    assert oracle.cycle_change(w, T) == pytest.approx(0.03, rel=1e-12)


def test_only_last_two_beats_count():
    T = 250

    def fn(t, k, col):
        base = np.sin(2 * np.pi * t / T)
        return np.where(t < T, 3.0 * base, base)      # the first beat differs, the last three agree

    w = _record(T, 4, 1, fn)
    assert oracle.cycle_change(w, T) < 1e-13
    assert oracle.cycle_change(w[: 2 * T], T) == pytest.approx(2.0 / 3.0, rel=1e-12)   # |1 - 3| / |3|


def test_short_record():
    T = 100
    w = _record(T, 2, 1, lambda t, k, col: np.sin(t))
    assert oracle.cycle_change(w[:-1], T) == -1.0
    assert oracle.cycle_change(w, T) >= 0.0
