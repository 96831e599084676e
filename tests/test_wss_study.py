"""Host logic of the wall-shear study: the wall-adjacent cell set and the
beat statistics (no GPU)."""
import numpy as np

import oracle
from paper_2112_05258_gb300 import wss_study
from workloads import configs


def test_wall_adjacent_cells_are_where_the_oracle_has_wss():
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    o = oracle.Oracle(inst)
    o.step(50)
    at = np.flatnonzero(np.abs(o.wall_shear()).sum(axis=1) > 0)
    at = at[(at // 256 >= 1) & (at // 256 <= 22)]
    assert np.array_equal(np.sort(wss_study._wall_adjacent(inst.node, 1, 22)), at)


def test_beat_statistics():
    # steady axial traction: OSI 0, no retrograde; a pure reversal: OSI 1/2
    ph = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    steady = np.zeros((64, 5, 3))
    steady[:, :, 2] = 1e-4
    osc = np.zeros((64, 5, 3))
    osc[:, :, 2] = 1e-4 * np.sin(ph)[:, None]
    for tv, osi, retro in ((steady, 0.0, 0.0), (osc, 0.5, 0.5)):
        ta = tv[:, :, 2]
        series = np.stack([ta.mean(axis=1), (ta < 0).mean(axis=1)], axis=1)
        s = wss_study._summary(series, ta, tv)
        assert abs(s["osi"] - osi) < 1e-12
        assert abs(s["beat_mean_retrograde_fraction"] - retro) < 0.02
