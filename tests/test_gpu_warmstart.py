"""The learned warm start against the cold-started method (small, quick case:
short beats, small tubes).  The network is trained on periodic states the
batched solver produced; on held-out parameter sets the warm-started runs
must become periodic in fewer beats than cold starts, and reach the same
periodic waveforms (the cold method is the judge)."""
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
    res = warmstart.evaluate(insts, pte, predict, precision_warm="f16")
    cold = np.array(res["cold_f32"]["cycles"])
    warm = np.array(res["warm_f32"]["cycles"])
    assert (cold > 0).all() and (warm > 0).all()
    assert np.median(warm) < np.median(cold)
    assert res["warm_f32"]["waveform_diff_vs_cold_median"] < 0.02
    assert res["warm_f16"]["waveform_diff_vs_cold_median"] < 0.02
