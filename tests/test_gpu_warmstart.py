"""The learned warm start against the cold-started method (small, quick case:
short beats, small tubes).  The network is trained on periodic states the
batched solver produced; on held-out parameter sets the warm-started runs
must become periodic in fewer beats than cold starts, and reach the same
periodic waveforms (the cold method is the reference)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_saves_beats():
    from paper_2112_05258_gb300 import load, warmstart
    from workloads import configs
    load()
    kw = dict(radius=4.0, length=32, period_range=(400, 800), kappa=configs.LV_KAPPA * 4000 / 600)
    _, ptr, ytr, cyc = warmstart.generate(256, 11, **kw)
    assert (cyc > 0).mean() > 0.9
    predict = warmstart.train(ptr, ytr, epochs=250, batch=256)
    insts, pte, yte, _ = warmstart.generate(32, 12, **kw)
    res = warmstart.evaluate(insts, pte, predict, precision_warm="f16", batch_size=16)   # two batches
    cold = np.array(res["cold_f32"]["cycles"])
    warm = np.array(res["warm_f32"]["cycles"])
    assert cold.size == 32 and len(res["cold_f32"]["steps"]) == 2
    assert (cold > 0).all() and (warm > 0).all()
    assert np.median(warm) < np.median(cold)
    assert res["warm_f32"]["waveform_diff_vs_cold_median"] < 0.02
    assert res["warm_f16"]["waveform_diff_vs_cold_median"] < 0.02


def test_warm_start_over_tube_sizes():
    # radius and length drawn per instance (inputs log R and log L besides the
    # six 0D parameters): small tubes of radius 3.5 .. 6 and length 24 .. 48
    from paper_2112_05258_gb300 import load, warmstart
    from workloads import configs
    load()
    kw = dict(period_range=(400, 800), kappa=configs.LV_KAPPA * 4000 / 600, geometry_sweep=True,
              radius_range=(3.5, 6.0), length_range=(24, 48))
    _, ptr, ytr, cyc = warmstart.generate(256, 21, keep_instances=False, batch_size=128, **kw)
    assert ptr.shape[1] == 8 and np.unique(ptr[:, 6]).size > 100 and (cyc > 0).mean() > 0.9
    predict = warmstart.train(ptr, ytr, epochs=250, batch=256)
    insts, pte, yte, _ = warmstart.generate(32, 22, **kw)
    assert len({i.shape for i in insts}) > 8
    res = warmstart.evaluate(insts, pte, predict, precision_warm="f16", batch_size=16)   # two batches
    cold = np.array(res["cold_f32"]["cycles"])
    warm = np.array(res["warm_f32"]["cycles"])
    assert cold.size == 32 and len(res["cold_f32"]["steps"]) == 2
    assert (cold > 0).all() and (warm > 0).all()
    assert np.median(warm) < np.median(cold)
    assert res["warm_f32"]["waveform_diff_vs_cold_median"] < 0.02
