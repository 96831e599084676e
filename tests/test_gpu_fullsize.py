"""Full-size parity: the aorta workload (128x128x1024, 4.0M fluid cells,
204,566 wall nodes, LV inlet, three RCR outlets) in the launch configuration
bench.py times (FP32, CUDA graphs, default block and occupancy variant)
against the FP64 oracle, from rest, over 20 steps -- long enough for the
ventricle to open its valve and drive flow into the lattice and for the wall
nodes to respond.  Every fluid cell's pressure and momentum, the waveforms of
all four boundaries and every wall node's position are compared."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_aorta_full_size_against_oracle():
    from paper_2112_05258_gb300 import Lattice, load
    from workloads import aorta
    load()
    inst = aorta.build(0)
    steps = 20
    lat = Lattice([inst], precision="f32", graph_steps=4)
    lat.step(steps)
    lat.sync()
    P, jx, jy, jz = lat.fields(0)
    wg = lat.waves(0)
    Xg = lat.ib_state(0, inst.ib.n)[0]
    o = oracle.Oracle(inst)
    o.step(steps)
    Po, jxo, jyo, jzo = o.macros()
    fl = inst.node.reshape(-1) == 0
    # FP32 storage of deviations: pressure to ~1e-7 of P_ref, momentum to
    # ~1e-5 of its largest value after 20 steps
    assert np.abs(P[fl] - Po[fl]).max() < 1e-6
    jmax = max(np.abs(jxo[fl]).max(), np.abs(jyo[fl]).max(), np.abs(jzo[fl]).max())
    assert jmax > 1e-6                          # the inflow has started
    for a, b in ((jx, jxo), (jy, jyo), (jz, jzo)):
        assert np.abs(a[fl] - b[fl]).max() < 1e-4 * jmax
    wo = o.waves()
    assert np.array_equal(wg[:, 0], wo[:, 0])
    for c in range(1, wo.shape[1]):
        scale = np.abs(wo[:, c]).max()
        if scale > 0:
            assert np.abs(wg[:, c] - wo[:, c]).max() < 1e-4 * scale + 1e-12
    Xo = o.ib_state()[0]
    assert np.abs(Xg - Xo).max() < 1e-7
