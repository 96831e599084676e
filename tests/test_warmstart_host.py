"""Host logic of the learned warm start (no GPU): the radial Legendre basis
against numpy's own Legendre series, the label read-out (mean gauge
pressures, area-mean velocities, least-squares modes) and the field layout
that applies a label, checked by reading the label back (a stand-in lattice
records what the warm start writes)."""
import numpy as np
import pytest

from paper_2112_05258_gb300 import warmstart as ws
from workloads import configs


def test_legendre_basis_matches_numpy():
    s = np.linspace(0.0, 1.0, 41)
    B = ws.legendre_basis(s, 8)
    for k in range(8):
        e = np.zeros(k + 1)
        e[k] = 1.0
        assert np.allclose(B[:, k], np.polynomial.legendre.legval(2 * s - 1, e), atol=1e-14)


def test_features_are_the_log_and_linear_inputs():
    p = np.array([[0.05, 200.0, 1.0, 2.0, 0.06, 4000.0]])
    f = ws.features(p)
    assert np.allclose(f, [[np.log(0.05), np.log(200.0), 0.0, 2.0, 0.06, np.log(4000.0)]], atol=1e-15)


class _Recorder:
    """Holds the fields and 0D states a warm start writes and returns them."""

    def __init__(self, inst):
        self.inst = inst
        self.n = int(np.prod(inst.shape))
        self.state = {0: np.zeros(8), 1: np.zeros(8)}

    def init_equilibrium(self, q, P, vx, vy, vz):
        self.P, self.vx, self.vy, self.vz = (np.array(a, float) for a in (P, vx, vy, vz))

    def set_0d_state(self, q, bc, value, valve_open=0.0, Td=-1e300):
        if bc == 0:
            self.state[0][4], self.state[0][6] = value, valve_open
        else:
            self.state[1][4] = value

    def fields(self, q):
        return self.P, self.vx, self.vy, self.vz   # at equilibrium j = rho0 v

    def state_0d(self, q, bc):
        return self.state[bc]


def test_apply_then_read_label_round_trip():
    inst = configs.rigid_tube(16, 16, 20, radius=6.0)
    layers = ws.Layers(inst)
    rng = np.random.default_rng(4)
    label = np.zeros(ws.N_OUT)
    label[0], label[1], label[2] = 2e-3, 5e-3, 1.0       # chamber, ventricle, valve open
    label[3], label[4] = 4e-3, 1e-3                      # inlet / outlet mean gauge pressure
    label[7:7 + 2 * ws.N_MODES] = rng.normal(0.0, 1e-2, 2 * ws.N_MODES) / (1 + np.arange(2 * ws.N_MODES))
    lat = _Recorder(inst)
    ws.apply(lat, 0, inst, label, layers)
    # pressure linear along the tube between the two layers, no transverse velocity
    nx, ny, nz = inst.shape
    Pz = lat.P.reshape(nz, ny, nx)[:, 0, 0]
    assert Pz[1] == pytest.approx(1 / 3 + label[3], abs=1e-15)
    assert Pz[nz - 2] == pytest.approx(1 / 3 + label[4], abs=1e-15)
    assert np.allclose(np.diff(Pz[1:nz - 1]), (label[4] - label[3]) / (nz - 3), atol=1e-15)
    assert not lat.vx.any() and not lat.vy.any()
    back = ws.read_label(lat, 0, layers)
    assert back[0] == label[0] and back[1] == label[1] and back[2] == label[2]
    assert back[3] == pytest.approx(label[3], abs=1e-15) and back[4] == pytest.approx(label[4], abs=1e-15)
    # the modes fitted at the layer cells are the ones applied
    assert np.allclose(back[7:7 + 2 * ws.N_MODES], label[7:7 + 2 * ws.N_MODES], atol=1e-12)
    # area-mean velocity of each layer: the mean of u / (P / c_s^2) over its cells
    for side, k in ((0, 5), (1, 6)):
        idx = layers.idx[side]
        assert back[k] == pytest.approx((lat.vz[idx] / (3 * lat.P[idx])).mean(), rel=1e-12)


def test_layers_are_the_first_fluid_layers():
    inst = configs.rigid_tube(16, 16, 20, radius=6.0)
    layers = ws.Layers(inst)
    nx, ny, nz = inst.shape
    for side, z in ((0, 1), (1, nz - 2)):
        idx = layers.idx[side]
        assert np.all(idx // (nx * ny) == z)
        assert idx.size == int((inst.node[z] == 0).sum())
        assert layers.s[side].max() <= 1.0 + 1e-12 and layers.s[side].min() >= 0.0
