"""Wall shear stress in the aorta workload at normal and high LV contractility
(the case study of Section 3.2, qualitatively: its geometry and data are not
published).

Both cases keep the beat period (so the Womersley number) and differ only in
the end-systolic elastance: E_max = 2.0 (normal) and 2.0 x 2.75 / 1.76
(high; the ratio of the two E_es values of Section 3.2), in the lattice
scaling of the aorta workload.  After ``beats - 1`` beats from rest the last
beat is sampled every ``every`` steps at a ring of the vessel between its
midpoint and outlet (cell heights z0 +- half_width, z0 = 0.75 nz):

* ``rigid``: the aorta with rigid walls (no membrane; the bounce-back wall
  sits at r = R(z) + 3).  WSS at the wall-adjacent fluid cells from the
  non-equilibrium stress (``Lattice.wall_shear``), projected on the local
  centreline tangent (axial WSS, positive downstream).
* ``ib``: the aorta with its elastic membrane.  The wall's shear is the
  tangential traction the fluid exerts on each membrane node, -F (the
  penalty force per area of Eq. LagForce acts on the fluid with +F),
  projected on the centreline tangent.

``--tau`` and ``--period`` change the viscosity and the beat (the elastance
scale and the Windkessel compliances follow the beat) to reach the paper's
Womersley number 16 at the ring, which the workload's tau = 0.8 and
4000-step beat (Womersley number about 3.5 there) do not.

Per sample: the ring mean of the axial WSS and the fraction of the ring
with negative (retrograde) axial WSS.  Per beat: minimum of the ring mean,
peak retrograde fraction, time-averaged WSS magnitude (TAWSS) and the
oscillatory shear index OSI = (1 - |mean tau| / mean |tau|) / 2, averaged
over the ring.

    python -m paper_2112_05258_gb300.wss_study --beats 3 --every 40 --out wss.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

E_NORMAL = 2.0
E_HIGH = 2.0 * 2.75 / 1.76


def _tangent(xc, yc):
    t = np.stack([np.gradient(xc), np.gradient(yc), np.ones_like(xc)], axis=1)
    return t / np.linalg.norm(t, axis=1, keepdims=True)


def _summary(series, tau_t, tau_vec):
    """series: (samples, 2) ring mean and retrograde fraction; tau_t:
    (samples, points) axial WSS; tau_vec: (samples, points, 3)."""
    mean_vec = tau_vec.mean(axis=0)
    mean_mag = np.linalg.norm(tau_vec, axis=2).mean(axis=0)
    osi = 0.5 * (1.0 - np.linalg.norm(mean_vec, axis=1) / np.maximum(mean_mag, 1e-300))
    return {
        "min_ring_mean_axial_wss": float(series[:, 0].min()),
        "max_ring_mean_axial_wss": float(series[:, 0].max()),
        "peak_retrograde_fraction": float(series[:, 1].max()),
        "beat_mean_retrograde_fraction": float(series[:, 1].mean()),
        "tawss": float(mean_mag.mean()),
        "osi": float(osi.mean()),
        "points": int(tau_t.shape[1]),
    }


def run_case(e_max: float, wall: str, beats: int, every: int, seed: int, z0: int | None,
             half_width: int, precision: str, tau: float | None = None, period: int | None = None):
    from workloads import aorta, configs
    from workloads.spec import BC_RCR
    from . import Lattice

    inst = aorta.build(seed, with_ib=(wall == "ib"))
    base = int(inst.boundaries[0].params[0])
    period = base if period is None else int(period)
    if tau is not None:
        inst.tau = float(tau)
    # a shorter beat keeps the stroke and the Windkessel time constants in
    # proportion: elastance scale x base/period, compliances x period/base
    inst.boundaries[0] = configs.lv_boundary(period=period, e_max=e_max,
                                             kappa=configs.LV_KAPPA * base / period)
    for b in inst.boundaries[1:]:
        if b.kind == BC_RCR:
            b.params[1] *= period / base
    nx, ny, nz = inst.shape
    z0 = int(0.75 * nz) if z0 is None else z0
    nu = (inst.tau - 0.5) / 3.0
    womersley = float(aorta.radius(nz)[z0] * np.sqrt(2 * np.pi / period / nu))
    xc, yc = aorta.centreline(seed, nz)
    tang = _tangent(xc, yc)
    lat = Lattice([inst], precision=precision, graph_steps=every if every <= 64 else 64,
                  wave_capacity=period)
    t0 = time.time()
    lat.step((beats - 1) * period)
    if wall == "rigid":
        cells = _wall_adjacent(inst.node, z0 - half_width, z0 + half_width)
        t_pts = tang[cells // (nx * ny)]
    else:
        n_ib = inst.ib.n
        zr = np.floor(inst.ib.X0[:, 2]).astype(int)
        nodes = np.flatnonzero(np.abs(zr - z0) <= half_width)
        t_pts = tang[zr[nodes]]
        rad = _radial(inst, nodes, xc, yc)
    series, taus_t, taus_v = [], [], []
    for s in range(period // every):
        lat.step(every)
        if wall == "rigid":
            tv = lat.wall_shear(0)[cells]
        else:
            F = lat.ib_state(0, n_ib)[2]
            tv = -F[nodes]
            tv = tv - np.sum(tv * rad, axis=1, keepdims=True) * rad     # tangential part
        ta = np.sum(tv * t_pts, axis=1)
        series.append([ta.mean(), float((ta < 0).mean())])
        taus_t.append(ta)
        taus_v.append(tv)
    lat.sync()
    wall_s = time.time() - t0
    waves = lat.waves(0)
    lat.close()
    series = np.asarray(series)
    out = _summary(series, np.asarray(taus_t), np.asarray(taus_v))
    out.update({
        "e_max": e_max, "wall": wall, "ring_z": [z0 - half_width, z0 + half_width],
        "tau": inst.tau, "period": period, "womersley": womersley,
        "inlet_peak_Qu": float(waves[:, 1].max()), "inlet_mean_Qu": float(waves[:, 1].mean()),
        "outlet_mean_Pbar": float(waves[:, 6].mean()),
        "phase": [(s + 1) * every / period for s in range(len(series))],
        "ring_mean_axial_wss": series[:, 0].tolist(),
        "retrograde_fraction": series[:, 1].tolist(),
        "seconds": wall_s,
    })
    return out


def _wall_adjacent(node, z_lo, z_hi):
    """Flat box indices of the fluid cells in heights [z_lo, z_hi] with a
    rigid-wall node (or the box edge) at one of their 18 lattice neighbours."""
    nz, ny, nx = node.shape
    pad = np.pad(node[z_lo - 1:z_hi + 2], ((0, 0), (1, 1), (1, 1)), constant_values=1)
    core = pad[1:-1, 1:-1, 1:-1]
    near = np.zeros(core.shape, bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) in (1, 2):
                    near |= pad[1 + dz:pad.shape[0] - 1 + dz, 1 + dy:pad.shape[1] - 1 + dy,
                                1 + dx:pad.shape[2] - 1 + dx] == 1
    z, y, x = np.nonzero((core == 0) & near)
    return (x + nx * (y + ny * (z + z_lo))).astype(np.int64)


def _radial(inst, nodes, xc, yc):
    X = inst.ib.X0[nodes]
    zr = np.floor(X[:, 2]).astype(int)
    r = np.stack([X[:, 0] - xc[zr], X[:, 1] - yc[zr], np.zeros(len(nodes))], axis=1)
    return r / np.linalg.norm(r, axis=1, keepdims=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--beats", type=int, default=3)
    ap.add_argument("--every", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--z0", type=int, default=None)
    ap.add_argument("--half-width", type=int, default=4)
    ap.add_argument("--walls", default="rigid,ib")
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--period", type=int, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = []
    for wall in a.walls.split(","):
        for name, e in (("normal", E_NORMAL), ("high", E_HIGH)):
            r = run_case(e, wall, a.beats, a.every, a.seed, a.z0, a.half_width, a.precision,
                         a.tau, a.period)
            r["case"] = name
            res.append(r)
            print(json.dumps({k: v for k, v in r.items() if not isinstance(v, list)}), flush=True)
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as f:
            json.dump(res, f)
    return res


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
