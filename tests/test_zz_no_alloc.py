"""lbm_boundary_flux_noalloc against the handle-based path.

The allocation-free entry point exists for callers whose device memory is
owned by their own allocator, or whose call site must not allocate; its
scratch is a fixed static device array.  This test feeds it the FP64 fields
of a running lattice (held in caller-owned torch tensors) and checks the
boundary flow and mean pressure it returns against the values the lattice's
own boundary kernels computed for the same time level (lbm_read_0d_state),
on two calls in a row so that the second call runs on scratch left by the
first.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu


def test_noalloc_flux_matches_boundary_state():
    torch = pytest.importorskip("torch")
    from paper_2112_05258_gb300 import Lattice, load
    L = load()
    inst = configs.rigid_tube(16, 16, 24, radius=5.0, period=200)
    nx, ny, nz = inst.shape
    lat = Lattice([inst], precision="f64")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    layers = ((1, +1), (nz - 2, -1))         # first fluid layers of inlet and outlet
    calls = 0
    for steps in (49, 29):
        lat.step(steps)
        P, jx, jy, jz = lat.fields(0)          # f(t_n) with n = steps taken so far
        lat.step(1)                            # the boundary kernels reduce the same t_n
        for k, (z, sign) in enumerate(layers):
            cells = (np.flatnonzero(inst.node[z].reshape(-1) == 0) + z * nx * ny).astype(np.int32)
            Pd = torch.tensor(P, dtype=torch.float64, device=dev)
            jn = torch.tensor(sign * jz, dtype=torch.float64, device=dev)
            cd = torch.tensor(cells, device=dev)
            out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
            st = L.lbm_boundary_flux_noalloc(ctypes.c_void_p(Pd.data_ptr()), ctypes.c_void_p(jn.data_ptr()),
                                             ctypes.c_void_p(cd.data_ptr()), int(cells.size),
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert st == 0
            torch.cuda.synchronize(dev)
            Q, Pmean = out.cpu().numpy()
            ref = lat.state_0d(0, k)           # {t, Q, Q_u, Pbar - P_ref, ...}
            assert Q == pytest.approx(ref[1], rel=1e-12, abs=1e-15)
            assert Pmean - 1.0 / 3.0 == pytest.approx(ref[3], rel=1e-12, abs=1e-15)
            calls += 1
    assert calls == 4


def test_noalloc_flux_rejects_oversized_request():
    torch = pytest.importorskip("torch")
    from paper_2112_05258_gb300 import load
    L = load()
    dev = torch.device("cuda:0")
    x = torch.ones(4, dtype=torch.float64, device=dev)
    c = torch.zeros(4, dtype=torch.int32, device=dev)
    p = ctypes.c_void_p
    assert L.lbm_boundary_flux_noalloc(p(x.data_ptr()), p(x.data_ptr()), p(c.data_ptr()), (1 << 20) + 1,
                                       p(x.data_ptr()), None) == -1
    assert L.lbm_boundary_flux_noalloc(p(x.data_ptr()), p(x.data_ptr()), p(c.data_ptr()), 0,
                                       p(x.data_ptr()), None) == -1
