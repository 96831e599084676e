"""GPU path (liblbm through its C-ABI) against the CPU oracle on identical
seeded inputs.

* FP64 instantiation: populations, macroscopic fields, 0D states and
  waveforms agree with the oracle to rounding (1e-12 absolute on f ~ 1/3,
  i.e. ~1e-11 relative to the deviations), over several 32-cell chunks and
  ragged row tails, for every boundary kind and the immersed boundary.
* FP32 on the rigid-tube workload (24x24x64, Womersley inlet, RCR outlet):
  pressure and flow waveforms within 1e-5 relative (max over time of the
  difference over the waveform's peak) after 10^4 steps.
"""
import numpy as np
import pytest

import oracle
from workloads import Instance, configs, geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lattice():
    from paper_2112_05258_gb300 import Lattice as L, load
    load()
    return L


def run_gpu(Lattice, inst, steps, prec="f64", f0=None, **kw):
    lat = Lattice([inst], precision=prec, **kw)
    if f0 is not None:
        lat.init_populations(0, f0)
    lat.step(steps)
    lat.sync()
    return lat


def run_oracle(inst, steps, f0=None):
    o = oracle.Oracle(inst)
    if f0 is not None:
        o.set_populations(f0)
    o.step(steps)
    return o


def assert_same(lat, o, inst, atol_f=1e-12, atol_w=1e-12):
    fl = inst.node.reshape(-1) == 0
    fg, fo = lat.populations(0), o.populations()
    assert np.abs(fg[:, fl] - fo[:, fl]).max() < atol_f
    mg, mo = lat.fields(0), o.macros()
    for a, b in zip(mg, mo):
        assert np.abs(a[fl] - b[fl]).max() < atol_f
    wg, wo = lat.waves(0), o.waves()
    assert wg.shape == wo.shape
    assert np.array_equal(wg[:, 0], wo[:, 0])
    if wg.shape[1] > 1:
        assert np.abs(wg[:, 1:] - wo[:, 1:]).max() < atol_w
    for k in range(len(inst.boundaries)):
        sg, so = lat.state_0d(0, k), o.state_0d(k)
        assert sg[0] == so[0] and sg[6] == so[6] and sg[7] == so[7]
        assert np.allclose(sg[1:6], so[1:6], rtol=1e-10, atol=1e-14)


def test_f64_closed_box_random(Lattice):
    inst = Instance(node=geometry.closed_box(37, 11, 9), tau=0.7)   # rows of 35: ragged chunks
    f0 = configs.random_populations(inst, seed=11, amp=1e-2)
    lat = run_gpu(Lattice, inst, 150, f0=f0)
    o = run_oracle(inst, 150, f0=f0)
    assert_same(lat, o, inst)


def test_f64_rigid_tube_womersley_rcr(Lattice):
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    f0 = configs.random_populations(inst, seed=3, amp=1e-3)
    lat = run_gpu(Lattice, inst, 300, f0=f0)
    o = run_oracle(inst, 300, f0=f0)
    assert_same(lat, o, inst)


def test_f64_lv_tube_along_x(Lattice):
    # the 0D boundaries on x: every row of the vessel begins and ends with a
    # boundary node, and the extrapolation links run along the rows
    inst = configs.lv_tube_x(30)
    f0 = configs.random_populations(inst, seed=11)
    assert_same(run_gpu(Lattice, inst, 300, f0=f0), run_oracle(inst, 300, f0=f0), inst)


def test_f64_pressure_tube(Lattice):
    inst = configs.pressure_tube(14, 14, 20, 4.5, 0.9, 2e-3, -1e-3)
    lat = run_gpu(Lattice, inst, 200)
    o = run_oracle(inst, 200)
    assert_same(lat, o, inst)


@pytest.mark.parametrize("order", [1, 2, 4])
def test_f64_lv_hybrid_inlet(Lattice, order):
    # several beats: the valve opens and closes, T_d and the smoothed closure
    # velocity are exercised; both 0D models marched at the given order
    inst = configs.lv_tube(period=600)
    for b in inst.boundaries:
        b.params = list(b.params[:4]) + [float(order)]
    lat = run_gpu(Lattice, inst, 1500)
    o = run_oracle(inst, 1500)
    w = o.waves()
    assert (np.diff(w[:, 4]) < 0).sum() >= 2        # at least two closures seen
    assert_same(lat, o, inst, atol_f=1e-11, atol_w=1e-11)
    if order == 1:
        assert_same_wss(lat, o, inst, 1e-12)


def assert_same_wss(lat, o, inst, atol):
    wg, wo = lat.wall_shear(0), o.wall_shear()
    at = np.abs(wo).sum(axis=1) > 0
    assert at.sum() > 0
    assert np.array_equal(at, np.abs(wg).sum(axis=1) > 0)
    assert np.abs(wg - wo).max() < atol


@pytest.mark.parametrize("filaments", [False, True])
def test_f64_immersed_boundary(Lattice, filaments):
    # spring wall, or the SGFD filament wall (31 axial filaments of 22 nodes)
    inst = configs.ib_tube(filaments=filaments)
    lat = run_gpu(Lattice, inst, 300)
    o = run_oracle(inst, 300)
    assert_same(lat, o, inst)
    n = inst.ib.n
    for a, b in zip(lat.ib_state(0, n), o.ib_state()):
        assert np.abs(a - b).max() < 1e-12
    assert_same_wss(lat, o, inst, 1e-12)        # band cells carry b in sigma


def test_filament_config_is_validated(Lattice):
    from paper_2112_05258_gb300 import LBMError
    for bad in ("end_unpinned", "repeated", "short"):
        inst = configs.ib_tube(filaments=True)
        fil = [f.copy() for f in inst.ib.filaments]
        if bad == "end_unpinned":
            inst.ib.pinned = inst.ib.pinned.copy()
            inst.ib.pinned[fil[0][-1]] = 0
        elif bad == "repeated":
            fil[1] = fil[1].copy()
            fil[1][3] = fil[0][3]
        else:
            fil[0] = fil[0][:2]
        inst.ib.filaments = fil
        with pytest.raises(LBMError):
            Lattice([inst], precision="f64")


def test_f32_wall_shear_rigid_tube(Lattice):
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    lat = run_gpu(Lattice, inst, 400, prec="f32")
    o = run_oracle(inst, 400)
    wg, wo = lat.wall_shear(0), o.wall_shear()
    at = np.abs(wo).sum(axis=1) > 0
    assert np.abs(wg[at] - wo[at]).max() < 1e-3 * np.abs(wo).max() + 1e-9


def _wave_rel_err(wg, wo, nbc):
    errs = {}
    for k in range(nbc):
        for col, name in ((1, "Q"), (2, "P")):
            a, b = wg[:, 1 + 4 * k + col - 1], wo[:, 1 + 4 * k + col - 1]
            errs[f"{name}{k}"] = np.abs(a - b).max() / np.abs(b).max()
    return errs


def test_f32_rigid_tube_1e4_steps(Lattice):
    inst = configs.rigid_tube()      # 24x24x64, R = 8, tau = 0.8, Womersley 0.02, T = 1000, RCR
    steps = 10000
    lat = run_gpu(Lattice, inst, steps, prec="f32", wave_capacity=steps)
    o = run_oracle(inst, steps)
    errs = _wave_rel_err(lat.waves(0), o.waves(), 2)
    assert max(errs.values()) < 1e-5, errs


@pytest.mark.parametrize("prec,bound", [("f16", 5e-2), ("bf16", 2e-1)])
def test_reduced_precision_waveform_error(Lattice, prec, bound):
    inst = configs.rigid_tube()
    steps = 2000
    lat = run_gpu(Lattice, inst, steps, prec=prec)
    o = run_oracle(inst, steps)
    errs = _wave_rel_err(lat.waves(0), o.waves(), 2)
    print(prec, errs)
    assert max(errs.values()) < bound, errs


def test_batch_equals_single(Lattice):
    a = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    b = configs.lv_tube(period=600)
    c = configs.ib_tube()
    for prec in ("f32", "f64"):
        batch = Lattice([a, b, c], precision=prec)
        batch.step(400)
        batch.sync()
        for q, inst in enumerate((a, b, c)):
            single = run_gpu(Lattice, inst, 400, prec=prec)
            if inst.ib is None:      # same kernels, deterministic reductions: identical bits
                assert np.array_equal(batch.populations(q), single.populations(0))
                assert np.array_equal(batch.waves(q), single.waves(0))
            else:                    # spreading uses atomics: equal to rounding
                tol = 1e-6 if prec == "f32" else 1e-14
                assert np.abs(batch.populations(q) - single.populations(0)).max() < tol
                assert np.abs(batch.waves(q) - single.waves(0)).max() < tol


def test_graph_equals_direct_launches(Lattice):
    inst = configs.lv_tube(period=600)
    g = Lattice([inst], precision="f32", graph_steps=8)
    g.step(203)
    d = Lattice([inst], precision="f32")
    d.set_kernel_timing(True)
    d.step(203)
    n, ms = d.kernel_time()
    assert n == 203 and ms > 0
    assert np.array_equal(g.populations(0), d.populations(0))
    assert np.array_equal(g.waves(0), d.waves(0))


@pytest.mark.parametrize("filaments", [False, True])
def test_graph_equals_direct_launches_with_ib(Lattice, filaments):
    # the same kernels captured in graphs or launched one by one: only the
    # order of the spreading atomics may differ
    # (inside the graphs the band velocities of the next step run beside the
    # boundary kernels, as two lists: both are non-empty on this tube)
    inst = configs.ib_tube(filaments=filaments)
    for prec, tol in (("f64", 1e-14), ("f32", 1e-6)):
        g = Lattice([inst], precision=prec, graph_steps=8)
        info = g.info()
        assert info.graph_steps == 8 and info.launches_per_step == info.launches_first_step + 1
        g.step(203)
        d = Lattice([inst], precision=prec)
        d.set_kernel_timing(True)
        d.step(203)
        assert np.abs(g.populations(0) - d.populations(0)).max() < tol
        assert np.abs(g.waves(0)[:, 1:] - d.waves(0)[:, 1:]).max() < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6)])
def test_slab_pipeline_equals_serial_step(Lattice, prec, tol):
    # the wall-node exchange pipelined over 6 slabs of lattice planes on three
    # streams: the same kernels and arithmetic as the serial step, only the
    # order of the spreading atomics may differ
    inst = configs.ib_tube()
    a = Lattice([inst], precision=prec, ib_slabs=8)
    assert a.info().slabs == 6 and a.info().launches_per_step == 6 * 3 + 2
    a.step(203)
    b = Lattice([inst], precision=prec)
    assert b.info().slabs == 0
    b.step(203)
    assert np.abs(a.populations(0) - b.populations(0)).max() < tol
    assert np.abs(a.waves(0)[:, 1:] - b.waves(0)[:, 1:]).max() < tol
    n = inst.ib.n
    for x, y in zip(a.ib_state(0, n), b.ib_state(0, n)):
        assert np.abs(x - y).max() < tol


def test_unstable_state_is_reported(Lattice):
    from paper_2112_05258_gb300 import LBMError
    inst = Instance(node=geometry.closed_box(10, 10, 10), tau=0.52)
    f0 = configs.random_populations(inst, seed=1, amp=0.0)
    f0[1] += 0.4                     # a strong +x jet everywhere: |v| > 0.3
    lat = Lattice([inst], precision="f32")
    lat.init_populations(0, f0)
    lat.step(5)
    with pytest.raises(LBMError) as e:
        lat.sync()
    assert e.value.status == -4


def test_ib_kernel_variants_agree(Lattice):
    # patch kernel (default) and the per-node kernels with 1, 2 or 4 threads
    # per node: the same arithmetic, only the order of the force sums differs
    inst = configs.ib_tube()
    ref = Lattice([inst], precision="f64")
    ref.step(120)
    n = inst.ib.n
    for tpn in (1, 2, 4):
        lat = Lattice([inst], precision="f64", ib_threads_per_node=tpn)
        lat.step(120)
        assert np.abs(lat.populations(0) - ref.populations(0)).max() < 1e-13
        for a, b in zip(lat.ib_state(0, n), ref.ib_state(0, n)):
            assert np.abs(a - b).max() < 1e-13


def test_fields_device_matches_host(Lattice):
    torch = pytest.importorskip("torch")
    inst = configs.lv_tube(period=300)
    lat = Lattice([inst], precision="f32")
    lat.step(250)
    nz, ny, nx = inst.node.shape
    outs = [torch.full((nz * ny * nx,), 7.0, dtype=torch.float32, device="cuda:0") for _ in range(4)]
    torch.cuda.synchronize()
    lat.fields_device(0, *(t.data_ptr() for t in outs))
    lat.sync()
    host = lat.fields(0)
    for t, h in zip(outs, host):
        assert np.array_equal(t.cpu().numpy(), h.astype(np.float32))


def test_degenerate_instances(Lattice):
    # an instance without fluid, a single fluid cell and an ordinary tube in
    # one batch: the empty and single-cell ones stay at rest, the tube runs
    # exactly as it does alone
    empty = Instance(node=np.ones((4, 5, 6), np.uint8), tau=0.8)
    one = np.ones((3, 3, 3), np.uint8)
    one[1, 1, 1] = 0
    single = Instance(node=one, tau=0.7)
    tube = configs.lv_tube(period=300)
    lat = Lattice([empty, single, tube], precision="f64")
    lat.step(150)
    lat.sync()
    alone = Lattice([tube], precision="f64")
    alone.step(150)
    assert np.array_equal(lat.populations(2), alone.populations(0))
    assert np.array_equal(lat.waves(2), alone.waves(0))
    assert np.abs(lat.populations(0)).max() == 0.0
    P, jx, jy, jz = lat.fields(1)
    assert P[13] == pytest.approx(1 / 3, abs=1e-15) and max(abs(jx[13]), abs(jy[13]), abs(jz[13])) < 1e-16
    only_empty = Lattice([empty], precision="f32")
    only_empty.step(10)
    only_empty.sync()
    assert np.abs(only_empty.fields(0)[0]).max() == 0.0
