"""Storage precision on the full-size aorta workload: FP16 and BF16 deviation
storage against the FP64 instantiation (itself equal to the oracle to 1e-15
on every component) over two beats of 4000 steps.  The 0D waveforms (flow
and mean pressure of the inlet and the three outlets) are compared as
max over time of |difference| / max |waveform|; the numbers are printed."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_aorta_reduced_precision_waveforms():
    from paper_2112_05258_gb300 import Lattice, load
    from workloads import aorta
    load()
    inst = aorta.build(0)
    steps = 8000
    waves = {}
    for prec in ("f64", "f32", "f16", "bf16"):
        lat = Lattice([inst], precision=prec, wave_capacity=steps)
        lat.step(steps)
        lat.sync()
        waves[prec] = lat.waves(0)
        lat.close()
    ref = waves["f64"]
    errs = {}
    for prec in ("f32", "f16", "bf16"):
        w = waves[prec]
        errs[prec] = max(np.abs(w[:, c] - ref[:, c]).max() / np.abs(ref[:, c]).max()
                         for k in range(4) for c in (1 + 4 * k, 2 + 4 * k))
    print("aorta 2-beat waveform error vs FP64:", errs)
    assert errs["f32"] < 1e-3 and errs["f16"] < 5e-2 and errs["bf16"] < 3e-1
