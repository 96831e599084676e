"""The synthetic workloads follow their stated recipes (no GPU): the
full-size aorta (128 x 128 x 1024, radius 40 -> 24, centreline offsets
within +-16 cells, two radius-10 branches leaving at heights in [300, 700]
to the x faces, an LV inlet and three RCR outlets, about 2e5 membrane nodes
with tether stiffness in [0.5, 2] x nominal) and the 256-tube batch (radius
in [6, 20], length in [128, 512], box side ceil(2R + 4), E_max in [1.5, 3],
period in [2000, 6000], resistances within +-50 % of R_p = 0.05, R_d = 1,
compliance within +-50 % of 1.5 T / R_d)."""
import math

import numpy as np
import pytest

from workloads import aorta, batch
from workloads.spec import BC_LV, BC_RCR


@pytest.fixture(scope="module")
def inst():
    return aorta.build(0)


def test_aorta_recipe(inst):
    assert inst.shape == (128, 128, 1024)
    R = aorta.radius()
    assert R[0] == pytest.approx(40.0, abs=0.02) and R[-1] == pytest.approx(24.0, abs=0.02)
    xc, yc = aorta.centreline(0)
    assert np.abs(xc - 64).max() <= 16 and np.abs(yc - 64).max() <= 16
    kinds = [b.kind for b in inst.boundaries]
    assert kinds == [BC_LV, BC_RCR, BC_RCR, BC_RCR]
    # branch outlets on the x faces, the aortic outlet on the top face
    assert [(b.axis, b.sign) for b in inst.boundaries[1:]] == [(2, -1), (0, -1), (0, +1)]
    for k, face in ((2, inst.node[:, :, -1]), (3, inst.node[:, :, 0])):
        zz, yy = np.nonzero(face == 2 + k)
        assert zz.size > 0 and 300 - 11 <= zz.min() and zz.max() <= 700 + 11
        area = zz.size
        assert area == pytest.approx(math.pi * 10 ** 2, rel=0.1)
    ib = inst.ib
    assert 1.9e5 < ib.n < 2.2e5
    k = np.asarray(ib.ks) / aorta.AORTA_K
    assert k.min() >= 0.5 and k.max() <= 2.0 and 1.2 < k.mean() < 1.3
    # membrane on r = R(z) about the centreline, pinned end rings only
    X = np.asarray(ib.X0)
    z = (X[:, 2] - 0.5).astype(int)
    r = np.hypot(X[:, 0] - xc[z], X[:, 1] - yc[z])
    assert np.abs(r - R[z]).max() < 1e-9
    pinned = np.asarray(ib.pinned).astype(bool)
    assert set(np.unique(z[pinned])) == {1, 1022}


def test_batch_recipe():
    insts, params = batch.tube_batch(256, 0)
    assert len(insts) == 256 and params.shape == (256, 6)
    Rp, C, Rd, Emax, Emin, T = params.T
    assert (Rp >= 0.025 - 1e-12).all() and (Rp <= 0.075 + 1e-12).all()
    assert (Rd >= 0.5 - 1e-12).all() and (Rd <= 1.5 + 1e-12).all()
    assert (C / (1.5 * T / 1.0) >= 0.5 - 1e-12).all() and (C / (1.5 * T) <= 1.5 + 1e-12).all()
    assert (Emax >= 1.5).all() and (Emax <= 3.0).all() and (Emin == 0.06).all()
    assert (T >= 2000).all() and (T <= 6000).all()
    for q in (0, 17, 255):
        nz, ny, nx = insts[q].node.shape
        assert nx == ny and 128 <= nz <= 512
        R = (nx - 4) / 2.0
        assert 6.0 - 0.5 <= R <= 20.0
        assert [b.kind for b in insts[q].boundaries] == [BC_LV, BC_RCR]
