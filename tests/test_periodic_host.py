"""Host logic around the periodic-state criterion (no GPU): the stepping and
bookkeeping of ``run_to_periodic`` for instances of different beats, with a
stand-in lattice whose cycle-to-cycle change halves every beat, and the
error and order arithmetic of the axisymmetric convergence study."""
import math
import types

import numpy as np
import pytest

from paper_2112_05258_gb300 import e5_study
from paper_2112_05258_gb300.periodic import run_to_periodic


class _HalvingLattice:
    def __init__(self, periods, start=0):
        self.t = start
        self.periods = np.asarray(periods)
        self.calls = []

    def info(self):
        return types.SimpleNamespace(steps=self.t)

    def step(self, n):
        self.t += n

    def cycle_change(self, periods):
        self.calls.append(self.t)
        assert np.array_equal(periods, self.periods)
        beats = self.t // self.periods
        return np.where(beats >= 2, 0.5 ** beats, -1.0)


def test_each_instance_is_periodic_at_its_own_first_beat_below_tol():
    lat = _HalvingLattice([400, 600])
    cycles, steps = run_to_periodic(lat, [400, 600], tol=0.01, max_cycles=20)
    # 0.5^b <= 0.01 first at b = 7 for both; the run stops once the slower one is
    assert list(cycles) == [7, 7]
    assert steps == 7 * 600
    # the change is only asked for at beat ends of some instance, from two beats on
    assert all(t % 200 == 0 for t in lat.calls) and min(lat.calls) >= 800


def test_never_periodic_within_the_cap_and_a_resumed_run():
    lat = _HalvingLattice([500])
    cycles, steps = run_to_periodic(lat, [500], tol=1e-9, max_cycles=5)
    assert list(cycles) == [-1] and steps == 5 * 500
    # beats are counted from the step the call starts at
    lat = _HalvingLattice([500], start=1000)
    cycles, steps = run_to_periodic(lat, [500], tol=0.01, max_cycles=20)
    assert steps == cycles[0] * 500 and cycles[0] >= 2


def test_convergence_study_orders():
    # errors against the finest run that fall as n_d^-2 give order 2
    res = []
    for n_d in (20, 40, 80, 160):
        w = np.sin(np.linspace(0, 2 * np.pi, 50))
        res.append({"n_d": n_d, "p_in": list(w + (n_d / 20.0) ** -2 * 1e-2 - 160.0 ** -2 * 400 * 1e-2)})
    e5_study.errors(res)
    for r in res[:2]:
        assert r["order_to_next"]["p_in"] == pytest.approx(
            math.log(((r["n_d"] / 20.0) ** -2 - (160 / 20.0) ** -2) /
                     ((2 * r["n_d"] / 20.0) ** -2 - (160 / 20.0) ** -2)) / math.log(2.0), rel=1e-9)
    assert res[-1]["err"]["p_in"] == 0.0
