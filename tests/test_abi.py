"""The C-ABI library builds, loads and exports every entry point that
include/lbm.h declares; lbm_create rejects invalid configurations before
touching a GPU (so these run on CPU-only machines)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_05258_gb300 import build as b
    b.build()
    from paper_2112_05258_gb300 import lbm
    return lbm.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2112_05258_gb300 import axisym, lbm, mlp
    assert sorted(lbm.EXPORTS + mlp.EXPORTS + axisym.EXPORTS) == names
    axisym.load()


def _cfg(lbm, node, tau=0.8, bcs=(), precision=0, graph_steps=0):
    nz, ny, nx = node.shape
    flat = np.ascontiguousarray(node.reshape(-1), dtype=np.uint8)
    arr = (lbm.BoundaryDesc * max(1, len(bcs)))()
    keep = [flat, arr]
    for k, (kind, params, period, etab) in enumerate(bcs):
        p = np.asarray(params, dtype=np.float64)
        keep.append(p)
        arr[k].kind, arr[k].axis, arr[k].sign = kind, 2, 1 if k == 0 else -1
        arr[k].n_params, arr[k].params = p.size, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if etab is not None:
            keep.append(etab)
            arr[k].period = period
            arr[k].elastance = etab.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    inst = (lbm.InstanceDesc * 1)()
    inst[0].nx, inst[0].ny, inst[0].nz = nx, ny, nz
    inst[0].node = flat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    inst[0].tau = tau
    inst[0].q_scale = 1
    inst[0].n_bc = len(bcs)
    inst[0].bc = ctypes.cast(arr, ctypes.POINTER(lbm.BoundaryDesc))
    keep.append(inst)
    cfg = lbm.Config(precision=precision, n_instances=1,
                     inst=ctypes.cast(inst, ctypes.POINTER(lbm.InstanceDesc)), graph_steps=graph_steps)
    return cfg, keep


def _create(lib, cfg):
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
    assert not h.value
    return st


def test_create_rejects_invalid_configs(lib):
    from paper_2112_05258_gb300 import lbm
    from workloads import geometry
    node = geometry.straight_tube(10, 10, 12, 3.0)
    rcr = (1, [0.05, 200.0, 1.0, 0.0], 0, None)
    vel = (3, [0.0], 0, None)
    assert lib.lbm_create(None, ctypes.byref(ctypes.c_void_p())) == -1
    for kwargs in (dict(tau=0.5), dict(tau=0.3), dict(precision=7), dict(graph_steps=3),
                   dict(bcs=(rcr,)),                                    # node code 3 undeclared
                   dict(bcs=(vel, (1, [0.05, 0.0, 1.0, 0.0], 0, None))),  # C = 0
                   dict(bcs=(vel, (2, [100, 1e-3, 30, 1e-3], 50, np.ones((50, 2))))),  # period mismatch
                   dict(bcs=(vel, (1, [0.05], 0, None)))):              # too few params
        cfg, keep = _cfg(lbm, node, **kwargs)
        assert _create(lib, cfg) == -1, kwargs
    node2 = node.copy()
    node2[5, 5, 5] = 9
    cfg, keep = _cfg(lbm, node2, bcs=(vel, rcr))
    assert _create(lib, cfg) == -1


def test_axisymmetric_create_rejects_invalid_configs(lib):
    # validation happens before any CUDA call
    from paper_2112_05258_gb300 import LBMError, axisym
    from workloads import axisym as axw
    axisym.load()
    good = axw.lv_tube()
    for mutate in ("tau", "column", "code"):
        inst = axw.lv_tube()
        node = inst.node.copy()
        if mutate == "tau":
            inst.tau = 0.5
        elif mutate == "column":
            node[2, 5] = 2                 # a boundary node off its column
        else:
            node[2, 5] = 7                 # a code without a boundary
        inst.node = node
        with pytest.raises(LBMError) as e:
            axisym.AxiLattice(inst)
        assert e.value.status == -1        # LBM_ERR_ARG, not a CUDA failure
    assert good.node.shape == (8, 40)
