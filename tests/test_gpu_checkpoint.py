"""Checkpoint and exact resume through the C-ABI: a run split by a
checkpoint restored into a fresh handle continues the saved trajectory
(bitwise without the immersed boundary, to the order of its float atomics
with it); a checkpoint is refused by a handle of another configuration."""
import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lattice():
    from paper_2112_05258_gb300 import Lattice as L, load
    load()
    return L


def _split_run(Lattice, insts, prec, first, second, **kw):
    a = Lattice(insts, precision=prec, **kw)
    a.step(first + second)
    b = Lattice(insts, precision=prec, **kw)
    b.step(first)
    ck = b.checkpoint()
    b.close()
    c = Lattice(insts, precision=prec, **kw)
    c.restore(ck)
    c.step(second)
    a.sync()
    c.sync()
    return a, c


def test_resume_is_bitwise_without_ib(Lattice):
    insts = [configs.lv_tube(period=300), configs.rigid_tube(16, 16, 24, radius=5.0, period=200)]
    a, c = _split_run(Lattice, insts, "f32", 173, 227, graph_steps=16)
    for q in range(2):
        assert np.array_equal(a.populations(q), c.populations(q))
        assert np.array_equal(a.waves(q), c.waves(q))
        for k in range(2):
            assert np.array_equal(a.state_0d(q, k), c.state_0d(q, k))


def test_resume_with_filament_wall(Lattice):
    inst = configs.ib_tube(filaments=True)
    a, c = _split_run(Lattice, [inst], "f64", 120, 80)
    assert np.abs(a.populations(0) - c.populations(0)).max() < 1e-13
    for x, y in zip(a.ib_state(0, inst.ib.n), c.ib_state(0, inst.ib.n)):
        assert np.abs(x - y).max() < 1e-13


def test_checkpoint_of_another_configuration_is_refused(Lattice):
    from paper_2112_05258_gb300 import LBMError
    a = Lattice([configs.lv_tube()], precision="f32")
    a.step(10)
    ck = a.checkpoint()
    b = Lattice([configs.rigid_tube(16, 16, 24, radius=5.0, period=200)], precision="f32")
    with pytest.raises(LBMError):
        b.restore(ck)
    with pytest.raises(LBMError):
        a.restore(ck[:100])
