"""Self-convergence of the axisymmetric lattice with the resolutions of the
paper's straight-aorta study (Section 3.1.3), dx = D/20, D/32, D/64, D/100,
D/128, under diffusive scaling, plus the throughput of the axisymmetric
kernels on a large grid.  Two cases (workloads.axisym):

* ``conv``: a 4-diameter tube, Womersley inlet (Womersley number 4), RCR
  outlet -- the rigid lattice near its incompressible limit at every
  resolution;
* ``paper``: the 25-diameter aorta with the hybrid LV inlet at Womersley
  number 16.  With rigid walls the lattice's acoustic transit of the tube
  is 8.7 beats at D/20 and 1.35 beats at D/128 under diffusive scaling, so
  the resolutions solve different compressible problems; it is run to show
  that, not to measure an order.

Each resolution runs ``beats`` beats from rest; over the last beat the
boundary data and the area-weighted mean pressure at the midpoint
cross-section are sampled at equally spaced phases, in units of the problem
(velocity D/T, pressure rho (D/T)^2).  Errors are L-infinity over the phases
against the finest resolution, relative to its peak; the observed order
between two resolutions is log(e1/e2)/log(n2/n1).

    python -m paper_2112_05258_gb300.e5_study --out e5.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

RESOLUTIONS = (20, 32, 64, 100, 128)
CASES = {
    # builder, period, phases, beats, sampled waveform columns
    "conv": ("convergence_tube", "conv_period", 40, 8, {"Pin": 2, "Qout": 5, "Pout": 6}),
    "paper": ("straight_aorta", "e5_period", 50, 20, {"Qin": 1, "Pin": 2, "Pout": 6}),
}


def run(case: str, n_d: int, precision: str, beats=None):
    from workloads import axisym as axw
    from .axisym import AxiLattice
    build, period, n_ph, beats0, cols = CASES[case]
    beats = beats or beats0
    inst = getattr(axw, build)(n_d)
    T = getattr(axw, period)(n_d)
    nr, nx = inst.node.shape
    lat = AxiLattice(inst, precision=precision, wave_capacity=max(8192, 2 * T))
    t0 = time.time()
    lat.step((beats - 1) * T)
    lat.sync()
    dt, dx = 1.0 / T, 1.0 / n_d
    su, sp = dt / dx, (dt / dx) ** 2
    r = np.arange(nr) + 0.5
    xm = nx // 2
    fl = inst.node[:, xm] == 0
    mid = []
    for k in range(n_ph):            # phase k / n_ph of the last beat, then advance
        P = lat.fields()[0]
        mid.append(float(((P[:, xm] - 1.0 / 3.0) * r * fl).sum() / (r * fl).sum()))
        lat.step(T // n_ph)
    lat.sync()
    wall = time.time() - t0
    W = lat.waves()
    w, prev = W[-T:], W[-2 * T:-T]   # row m: boundary data of step (beats - 1) T + m
    idx = np.arange(n_ph) * (T // n_ph)
    out = dict(case=case, n_d=n_d, period=T, tau=inst.tau, nx=nx, nr=nr, beats=beats, seconds=wall,
               cycle_change=float(np.abs(w[:, 2] - prev[:, 2]).max() / np.abs(prev[:, 2]).max()),
               Pmid=(np.array(mid) / sp).tolist())
    for key, col in cols.items():
        out[key] = (w[idx, col] / (su if key.startswith("Q") else sp)).tolist()
    lat.sync()
    t1 = time.time()
    lat.step(2 * 64 * 8)
    lat.sync()
    out["ms_per_step"] = (time.time() - t1) * 1e3 / (2 * 64 * 8)
    out["mlups"] = nx * nr / out["ms_per_step"] / 1e3
    lat.close()
    return out


def errors(res):
    fine = res[-1]
    keys = [k for k in fine if isinstance(fine[k], list)]
    for r in res:
        r["err"] = {k: float(np.abs(np.array(r[k]) - np.array(fine[k])).max() / np.abs(np.array(fine[k])).max())
                    for k in keys}
    for i in range(len(res) - 2):
        a1, a2 = res[i], res[i + 1]
        a1["order_to_next"] = {k: math.log(a1["err"][k] / a2["err"][k]) / math.log(a2["n_d"] / a1["n_d"])
                               for k in keys if a1["err"][k] > 0 and a2["err"][k] > 0}


def throughput(n_d: int, steps: int):
    """FP32 steps per second of a large grid with CUDA events around graph
    launches (the collide kernel moves 2 x 9 x 4 B per node)."""
    import torch
    from workloads import axisym as axw
    from .axisym import AxiLattice
    inst = axw.straight_aorta(n_d)
    nr, nx = inst.node.shape
    stream = torch.cuda.Stream()
    lat = AxiLattice(inst, precision="f32", stream=stream.cuda_stream)
    lat.step(256)
    lat.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fluid = int((inst.node == 0).sum())
    lat.close()
    return dict(n_d=n_d, nx=nx, nr=nr, fluid_nodes=fluid, ms_per_step=ms, mlups=fluid / ms / 1e3,
                gbs_algorithmic=72.0 * fluid / (ms * 1e-3) / 1e9)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--cases", default="conv,paper")
    ap.add_argument("--precision", default="f64")
    ap.add_argument("--resolutions", default=",".join(map(str, RESOLUTIONS)))
    ap.add_argument("--throughput-nd", type=int, default=1024)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    report = {}
    for case in [c for c in a.cases.split(",") if c]:
        res = [run(case, int(n), a.precision) for n in a.resolutions.split(",")]
        errors(res)
        for r in res:
            print(json.dumps({k: v for k, v in r.items() if not isinstance(v, list)}), flush=True)
        report[case] = res
    thr = throughput(a.throughput_nd, 1024) if a.throughput_nd else None
    if thr:
        print(json.dumps(thr), flush=True)
    report["throughput"] = thr
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as f:
            json.dump(report, f)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
