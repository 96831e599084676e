"""The aorta workload run for its full length (ten 4000-step beats, 4e4 steps)
in each storage precision, with the cycle-to-cycle change of its 0D
waveforms after every beat and the time to a periodic state.

Workload: ``workloads.aorta.build(seed)`` (128 x 128 x 1024, 4.02M fluid
cells, LV elastance inlet with its valves, three RCR outlets, 204,566
elastic wall nodes), from rest.  After every beat b >= 2 the device computes
delta_b = max over the boundaries and the waveforms W in {Q_u, mean gauge
pressure} of max_t |W(t) - W(t - T)| / max_t |W(t - T)| over the last beat
(``Lattice.cycle_change``); the run counts as periodic at the first beat
with delta_b <= tol (1 %).  The wall time to that beat is the host clock
over the steps taken (the host waits for the device once per beat; the
read-outs between quarter beats are not timed).  Also recorded per beat: the
largest wall-node displacement component |X - X0|, sampled at every quarter
beat (a node that leaves its support box stops the run with the device
status word).

For each reduced precision the waveforms of the last beat are compared with
the FP32 run's (same metric: max over boundaries and waveforms of
max_t |W_p - W_FP32| / max_t |W_FP32|), the plain FP32 method being the reference.

    python -m paper_2112_05258_gb300.aorta_run --beats 10 --out aorta_run.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def last_beat(waves: np.ndarray, period: int) -> np.ndarray:
    """Q_u and mean gauge pressure of every boundary over the last beat:
    (period, 2 * n_bc) from rows {step, then per boundary Q_u, Pbar, state,
    valve}."""
    w = waves[-period:, 1:]
    nbc = w.shape[1] // 4
    cols = [4 * k + j for k in range(nbc) for j in (0, 1)]
    return w[:, cols]


def waveform_difference(a: np.ndarray, ref: np.ndarray) -> float:
    """max over waveforms of max_t |a - ref| / max_t |ref|."""
    scale = np.abs(ref).max(axis=0)
    scale[scale == 0] = 1.0
    return float((np.abs(a - ref).max(axis=0) / scale).max())


def run(inst, precision: str, beats: int, period: int, tol: float):
    from paper_2112_05258_gb300 import Lattice
    from paper_2112_05258_gb300.lbm import LBMError
    lat = Lattice([inst], precision=precision, wave_capacity=2 * period + 64)
    n_ib = inst.ib.X0.shape[0] if inst.ib is not None else 0
    delta, wall, disp, periodic_beat, periodic_s = [], [], [], -1, None
    t_total = 0.0
    quarters = [period // 4 + (1 if q < period % 4 else 0) for q in range(4)]
    for b in range(1, beats + 1):
        dmax = 0.0
        for n in quarters:
            t0 = time.perf_counter()
            lat.step(n)
            try:
                lat.sync()
            except LBMError as e:  # the device status word: the run left the stable range
                lat.close()
                return {"precision": precision, "failed_in_beat": b, "error": str(e),
                        "delta_per_beat": delta, "wall_s_per_beat": wall,
                        "max_wall_displacement_per_beat": disp}, None
            t_total += time.perf_counter() - t0
            if n_ib:  # largest component of X - X0 over the wall nodes, four times a beat
                X = lat.ib_state(0, n_ib)[0]
                dmax = max(dmax, float(np.abs(X - np.asarray(inst.ib.X0)).max()))
        wall.append(t_total)
        if n_ib:
            disp.append(dmax)
        d = float(lat.cycle_change([period])[0]) if b >= 2 else -1.0
        delta.append(d)
        if periodic_beat < 0 and 0 <= d <= tol:
            periodic_beat, periodic_s = b, t_total
    W = last_beat(lat.waves(0, max_rows=period), period)
    info = lat.info()
    lat.close()
    return {"precision": precision, "steps": beats * period, "wall_s": t_total,
            "mlups": info.fluid_cells * beats * period / t_total / 1e6,
            "delta_per_beat": delta, "wall_s_per_beat": wall, "max_wall_displacement_per_beat": disp,
            "periodic_beat": periodic_beat, "time_to_periodic_s": periodic_s}, W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--beats", type=int, default=10)
    ap.add_argument("--precisions", default="f32,f16,bf16")
    ap.add_argument("--tol", type=float, default=0.01)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from workloads import aorta
    period = 4000  # the workload's beat
    inst = aorta.build(args.seed, period=period)
    results, ref = [], None
    for p in args.precisions.split(","):
        r, W = run(inst, p, args.beats, period, args.tol)
        if p == "f32":
            ref = W
        elif ref is not None and W is not None:
            r["last_beat_vs_f32"] = waveform_difference(W, ref)
        results.append(r)
        print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"workload": f"aorta seed {args.seed}, beat {period} steps", "fluid_cells": inst.n_fluid,
                       "tol": args.tol, "runs": results}, f, indent=1)


if __name__ == "__main__":
    main()
