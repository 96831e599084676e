"""Self-convergence of the 3D coupled solver (the 3D analogue of the
paper's straight-tube convergence study, Section 3.1.3): the rigid tube of
the parity workload (24x24x64, R = 8, Womersley inlet with Womersley number
2, RCR outlet) at R = 4, 8, 16 under diffusive scaling (tau fixed, beat
~ R^2, velocity ~ 1/R, 0D parameters carried by the unit scales).  The
inlet pressure and flow waveforms over the last beat, in problem units,
converge to the finest grid at an order between 1 (the staircase wall) and
2 (the lattice)."""
import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu

N_PH = 50


def _case(R):
    s_u = 8.0 / R                   # (dt/dx) relative to R = 8
    s_c = R ** 3 / 512.0            # (dx/dt^2) relative to R = 8
    T = int(1000 * (R / 8) ** 2)
    n = 3 * R
    inst = configs.rigid_tube(n, n, 8 * R, radius=float(R), tau=0.8, u_peak=0.02 * s_u, period=T,
                              rcr=(0.05 * s_u, 200.0 * s_c, 1.0 * s_u, 0.0))
    return inst, T, s_u


def _waves(Lattice, R, beats=6):
    inst, T, s_u = _case(R)
    lat = Lattice([inst], precision="f64", wave_capacity=T)
    lat.step(beats * T)
    lat.sync()
    w = lat.waves(0)[-T:]
    idx = np.arange(N_PH) * (T // N_PH)
    return w[idx, 2] / s_u ** 2, w[idx, 1] / s_u       # inlet gauge pressure, inlet flow


def test_three_dimensional_self_convergence():
    from paper_2112_05258_gb300 import Lattice, load
    load()
    P, Q = {}, {}
    for R in (4, 8, 16):
        P[R], Q[R] = _waves(Lattice, R)
    for X in (P, Q):
        e4 = np.abs(X[4] - X[16]).max() / np.abs(X[16]).max()
        e8 = np.abs(X[8] - X[16]).max() / np.abs(X[16]).max()
        order = np.log(e4 / e8) / np.log(2.0)
        print(f"3D self-convergence: e(R=4) {e4:.4g} e(R=8) {e8:.4g} order {order:.3f}")
        assert e8 < e4 and 0.8 < order < 3.0, (e4, e8, order)
