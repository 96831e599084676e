"""GPU tests of the batching, periodic-state and initialisation entry points."""
import numpy as np
import pytest

import oracle
from workloads import batch, configs

pytestmark = pytest.mark.gpu
CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def Lattice():
    from paper_2112_05258_gb300 import Lattice as L, load
    load()
    return L


def _fields(inst):
    nx, ny, nz = inst.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x + 0.5 - nx / 2) ** 2 + (y + 0.5 - ny / 2) ** 2
    P = CS2 + 1e-3 * (1 - z / nz) + 2e-4 * np.sin(0.3 * x)
    uz = 0.01 * np.clip(1 - r2 / 25.0, 0, None)
    ux = 1e-3 * np.cos(0.2 * z)
    uy = np.zeros_like(uz)
    return [a.reshape(-1) for a in (P, ux, uy, uz)]


def test_init_equilibrium_matches_oracle(Lattice):
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    P, ux, uy, uz = _fields(inst)
    lat = Lattice([inst], precision="f64")
    lat.init_equilibrium(0, P, ux, uy, uz)
    f0 = np.stack([oracle.feq(P[c], [ux[c], uy[c], uz[c]]) for c in range(P.size)], axis=1)
    fl = inst.node.reshape(-1) == 0
    assert np.abs(lat.populations(0)[:, fl] - f0[:, fl]).max() < 1e-15
    o = oracle.Oracle(inst)
    o.set_populations(f0)
    lat.step(120)
    o.step(120)
    assert np.abs(lat.populations(0)[:, fl] - o.populations()[:, fl]).max() < 1e-12
    assert np.abs(lat.waves(0)[:, 1:] - o.waves()[:, 1:]).max() < 1e-12


def test_cycle_change_matches_waveforms(Lattice):
    periods = (600, 400, 500, 300)
    insts = [configs.lv_tube(period=T) for T in periods]
    lat = Lattice(insts, precision="f32", wave_capacity=4096)
    lat.step(900)
    d = lat.cycle_change(periods)
    assert d[0] == -1.0 and d[1] >= 0.0                 # instance 0 lacks two beats of history
    lat.step(1000)
    d = lat.cycle_change(periods)
    for q, T in enumerate(periods):
        # the oracle's criterion on the same (GPU) record
        assert d[q] == pytest.approx(oracle.cycle_change(lat.waves(q), T), rel=1e-12)


def test_cycle_change_matches_oracle_run(Lattice):
    """Periodic-state detection against the oracle: the FP64 instantiation
    and the CPU oracle run the same seeded LV tube; the device criterion on
    the device record equals the oracle's criterion on the oracle's record."""
    T = 300
    inst = configs.lv_tube(period=T)
    lat = Lattice([inst], precision="f64", wave_capacity=2048)
    o = oracle.Oracle(inst)
    lat.step(2 * T - 1)
    o.step(2 * T - 1)
    assert lat.cycle_change([T])[0] == -1.0 and oracle.cycle_change(o.waves(), T) == -1.0
    for more in (1, 157, 443):          # window aligned with the start of a beat, then not
        lat.step(more)
        o.step(more)
        d_orc = oracle.cycle_change(o.waves(), T)
        assert d_orc > 0.0
        assert lat.cycle_change([T])[0] == pytest.approx(d_orc, rel=1e-9)


def test_autotune_keeps_trajectory(Lattice):
    inst = configs.lv_tube(period=600)
    a = Lattice([inst], precision="f64")
    a.step(10)
    (block, minb, cpt), times = a.autotune(iters=3, return_times=True)
    assert block in (64, 128, 192, 256) and minb in (3, 4, 5, 6, 8) and cpt in (1, 2)
    assert times.shape == (5, 4) and (times > 0).all()
    a.step(190)
    b = Lattice([inst], precision="f64")
    b.step(200)
    assert np.abs(a.populations(0) - b.populations(0)).max() < 1e-15
    assert np.array_equal(a.waves(0), b.waves(0))


def test_set_0d_state_round_trip(Lattice):
    inst = configs.lv_tube(period=600)
    lat = Lattice([inst], precision="f32")
    lat.set_0d_state(0, 1, 0.0042)
    lat.set_0d_state(0, 0, 0.0031, valve_open=1.0, Td=-5.0)
    s1, s0 = lat.state_0d(0, 1), lat.state_0d(0, 0)
    assert s1[4] == 0.0042 and s0[4] == 0.0031 and s0[6] == 1.0 and s0[7] == -5.0


def test_run_to_periodic_small_batch(Lattice):
    from paper_2112_05258_gb300.periodic import run_to_periodic
    insts = [configs.lv_tube(period=T) for T in (400, 600)]
    lat = Lattice(insts, precision="f32", wave_capacity=4096)
    cycles, steps = run_to_periodic(lat, [400, 600], tol=0.01, max_cycles=30)
    assert (cycles > 1).all()
    d = lat.cycle_change([400, 600])
    assert (d <= 0.02).all()


def test_uneven_batch_equals_single(Lattice):
    insts, params = batch.tube_batch(6, seed=5)
    lat = Lattice(insts, precision="f32")
    lat.step(300)
    for q in (0, 3, 5):
        single = Lattice([insts[q]], precision="f32")
        single.step(300)
        assert np.array_equal(lat.populations(q), single.populations(0))
        assert np.array_equal(lat.waves(q), single.waves(0))


@pytest.mark.parametrize("variant", range(5))
def test_every_stream_collide_variant_gives_the_trajectory(Lattice, variant):
    # the occupancy and cells-per-thread variants run the same per-cell
    # arithmetic: the instance without wall nodes agrees bit for bit in FP32;
    # the second has wall nodes, whose spreading atomics add in run order, and
    # agrees to rounding under any variant
    insts = [configs.lv_tube(period=300), configs.ib_tube()]
    ref = Lattice(insts, precision="f64")
    ref.step(120)
    lat = Lattice(insts, precision="f64")
    lat.set_stream_collide_shape(96 if variant % 2 else 128, variant)
    lat.step(120)
    for q in range(2):
        assert np.abs(lat.populations(q) - ref.populations(q)).max() < 1e-14
        assert np.abs(lat.waves(q)[:, 1:] - ref.waves(q)[:, 1:]).max() < 1e-14
    tols = {"f16": (1e-6, 4e-5), "f32": (0.0, 2e-7)}
    for prec, tol in tols.items():
        a = Lattice(insts, precision=prec)
        a.set_stream_collide_shape(128, variant)
        a.step(60)
        b = Lattice(insts, precision=prec)
        b.step(60)
        for q in range(2):
            assert np.abs(a.populations(q) - b.populations(q)).max() <= tol[q], (prec, q)


def test_set_0d_params_is_stream_ordered(Lattice):
    # parameters set before the first step equal a lattice created with them
    # (and the oracle); set between queued steps they act from the next step
    # on, with or without the host waiting in between
    import oracle
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    new = [0.05, 120.0, 0.7, 0.0]
    inst2 = configs.rigid_tube(16, 16, 24, radius=5.0, period=200, rcr=tuple(new))
    a = Lattice([inst], precision="f64")
    a.set_0d_params(0, 1, new)
    a.step(150)
    o = oracle.Oracle(inst2)
    o.step(150)
    assert np.abs(a.waves(0)[:, 1:] - o.waves()[:, 1:]).max() < 1e-12
    queued = Lattice([inst], precision="f32", graph_steps=16)
    queued.step(100)
    queued.set_0d_params(0, 1, new)          # no wait for the 100 steps
    queued.step(100)
    waited = Lattice([inst], precision="f32", graph_steps=16)
    waited.step(100)
    waited.sync()
    waited.set_0d_params(0, 1, new)
    waited.step(100)
    plain = Lattice([inst], precision="f32", graph_steps=16)
    plain.step(200)
    wq, ww, wp = queued.waves(0), waited.waves(0), plain.waves(0)
    assert np.array_equal(wq, ww)
    assert np.array_equal(wq[:100], wp[:100]) and not np.array_equal(wq[100:], wp[100:])


def test_async_0d_state_read_equals_sync(Lattice):
    torch = pytest.importorskip("torch")
    insts = [configs.lv_tube(period=300), configs.rigid_tube(16, 16, 24, radius=5.0, period=200)]
    lat = Lattice(insts, precision="f32")
    bufs = [torch.zeros(8 * 2, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    for k in range(3):
        lat.step(37)
        lat.state_0d_async(k % 2, bufs[k].data_ptr())
    lat.sync()
    # the last read is of instance 0 after 111 steps
    got = bufs[2].numpy().reshape(2, 8)
    for bc in range(2):
        assert np.array_equal(got[bc], lat.state_0d(0, bc))
    assert bufs[0].numpy()[0] == 37.0 and bufs[1].numpy()[0] == 74.0


def test_async_0d_state_read_into_pageable_memory(Lattice):
    # memory the device cannot address goes through the device buffer and a
    # copy; the values are the same as the direct write into pinned memory
    torch = pytest.importorskip("torch")
    inst = configs.lv_tube(period=300)
    lat = Lattice([inst], precision="f32")
    lat.step(50)
    pinned = torch.zeros(16, dtype=torch.float64, pin_memory=True)
    pageable = np.zeros(16)
    lat.state_0d_async(0, pinned.data_ptr())
    lat.state_0d_async(0, pageable.ctypes.data)
    lat.sync()
    assert pageable[0] == 50.0 and np.array_equal(pageable, pinned.numpy())


def test_once_per_boundary_0d_step_equals_per_block(Lattice):
    # a batch whose link blocks exceed one wave (64 uneven LV tubes: about
    # 1,400 blocks) takes each boundary's 0D step once, in the last reduction
    # block to arrive; a single tube takes it in every link block.  The sums
    # and the step are the same arithmetic, so the bits agree.
    insts, _ = batch.tube_batch(64, 3)
    big = Lattice(insts, precision="f32", wave_capacity=512)
    big.step(150)
    big.sync()
    for q in (0, 17, 63):
        single = Lattice([insts[q]], precision="f32", wave_capacity=512)
        single.step(150)
        assert np.array_equal(big.waves(q), single.waves(0))
        assert np.array_equal(big.populations(q), single.populations(0))
        single.close()


def _step_io_case(Lattice, inst, prec, n, start):
    """Runs n steps of instance inst (after `start` plain steps) once through
    lbm_step_io and once as per-step host calls (set the outlet params, one
    step, asynchronous state read); returns both lattices and both row arrays."""
    import torch
    nbc = len(inst.boundaries)
    base = np.array(inst.boundaries[1].params, dtype=np.float64)
    params = torch.zeros((n, base.size), dtype=torch.float64, pin_memory=True)
    for k in range(n):  # a time-varying outlet resistance R_p
        params[k] = torch.from_numpy(base * np.array([1.0 + 0.3 * np.sin(2 * np.pi * k / 50.0)] +
                                                     [1.0] * (base.size - 1)))
    got = torch.full((n, 8 * nbc), -1.0, dtype=torch.float64, pin_memory=True)
    a = Lattice([inst], precision=prec)
    a.step(start)
    a.step_io(0, 1, n, params.data_ptr(), base.size, got.data_ptr())
    a.sync()
    want = torch.full((n, 8 * nbc), -1.0, dtype=torch.float64, pin_memory=True)
    b = Lattice([inst], precision=prec)
    b.step(start)
    for k in range(n):
        b.set_0d_params(0, 1, params[k].numpy())
        b.step(1)
        b.state_0d_async(0, want[k].data_ptr())
    b.sync()
    return a, b, got.numpy(), want.numpy()


def test_step_io_equals_per_step_calls(Lattice):
    # per-step params read and state rows written by the device inside the
    # step graphs (two graphs of 64 steps and a remainder of 22, starting at
    # an odd step) equal the per-step host calls bit for bit on an instance
    # without wall nodes; the rows carry consecutive step counts
    a, b, got, want = _step_io_case(Lattice, configs.lv_tube(period=300), "f64", 150, 7)
    assert np.array_equal(got, want)
    assert np.array_equal(got[:, 0], np.arange(8, 158))
    assert np.array_equal(a.populations(0), b.populations(0))
    assert np.array_equal(a.waves(0), b.waves(0))
    assert a.info().steps == b.info().steps == 157


def test_step_io_with_wall_nodes(Lattice):
    # with wall nodes the graphs also run the band velocities beside the
    # boundary kernels: equal to the per-step calls to the rounding of the
    # spreading atomics
    for prec, tol in (("f64", 1e-14), ("f32", 1e-6)):
        a, b, got, want = _step_io_case(Lattice, configs.ib_tube(), prec, 100, 3)
        assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max())
        assert np.abs(a.populations(0) - b.populations(0)).max() < tol


def test_step_io_rejects_bad_arguments(Lattice):
    import torch
    inst = configs.lv_tube(period=300)
    lat = Lattice([inst], precision="f64")
    rows = torch.zeros((4, 16), dtype=torch.float64, pin_memory=True)
    pageable = np.zeros((4, 4))
    pinned = torch.tensor(np.tile(inst.boundaries[1].params, (4, 1)), dtype=torch.float64).pin_memory()
    with pytest.raises(RuntimeError):  # params in pageable host memory
        lat.step_io(0, 1, 4, pageable.ctypes.data, 4, rows.data_ptr())
    bad = pinned.clone().pin_memory()
    bad[2, 1] = -1.0  # a compliance <= 0 in the third set
    with pytest.raises(RuntimeError):
        lat.step_io(0, 1, 4, bad.data_ptr(), 4, rows.data_ptr())
    assert lat.info().steps == 0  # nothing was enqueued
    lat.step_io(0, 1, 4, pinned.data_ptr(), 4, rows.data_ptr())
    lat.sync()
    assert lat.info().steps == 4
