"""Host logic of the full-length aorta study: the last-beat waveform
selection, the waveform difference, the periodic-beat bookkeeping and the
handling of a run stopped by the device status word (a stand-in lattice,
no GPU)."""
import types

import numpy as np
import pytest

import paper_2112_05258_gb300 as pkg
from paper_2112_05258_gb300 import aorta_run
from paper_2112_05258_gb300.lbm import LBMError


def test_last_beat_takes_flow_and_pressure_of_every_boundary():
    T, nbc = 7, 3
    w = np.arange(20 * (1 + 4 * nbc), dtype=float).reshape(20, 1 + 4 * nbc)
    lb = aorta_run.last_beat(w, T)
    assert lb.shape == (T, 2 * nbc)
    for k in range(nbc):
        assert np.array_equal(lb[:, 2 * k], w[-T:, 1 + 4 * k])      # Q_u
        assert np.array_equal(lb[:, 2 * k + 1], w[-T:, 2 + 4 * k])  # mean gauge pressure


def test_waveform_difference():
    t = np.linspace(0.0, 1.0, 50)
    ref = np.stack([np.sin(6.3 * t), 2.0 + np.cos(6.3 * t), np.zeros_like(t)], axis=1)
    assert aorta_run.waveform_difference(ref, ref) == 0.0
    # the worst waveform decides; each is scaled by its own maximum
    a = ref.copy()
    a[:, 1] += 0.03
    assert aorta_run.waveform_difference(a, ref) == pytest.approx(0.03 / 3.0)
    # an identically zero reference waveform is compared unscaled
    a = ref.copy()
    a[:, 2] = 1e-3
    assert aorta_run.waveform_difference(a, ref) == pytest.approx(1e-3)


class _FakeLattice:
    """Advances a step counter; cycle_change follows a given sequence per beat,
    sync fails past a given step, wall nodes drift by 1e-3 per step count."""

    deltas = None
    fail_after = None
    period = None

    def __init__(self, insts, precision="f32", wave_capacity=0):
        self.t = 0
        self.n_bc = 2
        self.closed = False

    def step(self, n):
        self.t += n

    def sync(self):
        if self.fail_after is not None and self.t > self.fail_after:
            raise LBMError(-4, "a wall node moved outside its immersed-boundary band")

    def ib_state(self, inst, n):
        X = np.full((n, 3), 1e-6 * self.t)
        return [X, X * 0, X * 0, X * 0]

    def cycle_change(self, periods):
        return np.array([self.deltas[self.t // self.period - 1]])

    def waves(self, inst, max_rows=1 << 30):
        rows = min(max_rows, self.t)
        w = np.zeros((rows, 1 + 4 * self.n_bc))
        w[:, 0] = np.arange(self.t - rows, self.t)
        w[:, 1] = np.sin(w[:, 0] / 10.0)
        return w

    def info(self):
        return types.SimpleNamespace(fluid_cells=1000)

    def close(self):
        self.closed = True


def _inst(n_nodes=4):
    return types.SimpleNamespace(ib=types.SimpleNamespace(X0=np.zeros((n_nodes, 3))))


def test_periodic_beat_is_the_first_at_or_below_tolerance(monkeypatch):
    T = 40
    fake = type("F", (_FakeLattice,), {"deltas": [-1, 1.0, 0.2, 0.011, 0.009, 0.02, 0.001],
                                       "fail_after": None, "period": T})
    monkeypatch.setattr(pkg, "Lattice", fake)
    r, W = aorta_run.run(_inst(), "f32", beats=7, period=T, tol=0.01)
    assert r["periodic_beat"] == 5  # later beats above the tolerance do not move it
    assert r["time_to_periodic_s"] == pytest.approx(r["wall_s_per_beat"][4])
    assert r["delta_per_beat"][0] == -1.0 and r["delta_per_beat"][4] == pytest.approx(0.009)
    assert r["steps"] == 7 * T and len(r["wall_s_per_beat"]) == 7
    # displacement: the largest of four samples a beat, i.e. the beat's end here
    assert r["max_wall_displacement_per_beat"][-1] == pytest.approx(1e-6 * 7 * T)
    assert W.shape == (T, 4)


def test_never_periodic_and_stopped_runs(monkeypatch):
    T = 40
    fake = type("F", (_FakeLattice,), {"deltas": [-1, 1.0, 0.5, 0.3], "fail_after": None, "period": T})
    monkeypatch.setattr(pkg, "Lattice", fake)
    r, _ = aorta_run.run(_inst(), "f16", beats=4, period=T, tol=0.01)
    assert r["periodic_beat"] == -1 and r["time_to_periodic_s"] is None
    # a status-word failure in the third beat ends the run with what was measured before it
    fake = type("F", (_FakeLattice,), {"deltas": [-1, 1.0, 0.5, 0.3], "fail_after": 2 * T + 5, "period": T})
    monkeypatch.setattr(pkg, "Lattice", fake)
    r, W = aorta_run.run(_inst(), "bf16", beats=4, period=T, tol=0.01)
    assert W is None
    assert r["failed_in_beat"] == 3 and "immersed-boundary band" in r["error"]
    assert len(r["delta_per_beat"]) == 2 and len(r["max_wall_displacement_per_beat"]) == 2
