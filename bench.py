#!/usr/bin/env python
"""Throughput of the full 0D-3D coupled lattice Boltzmann step on one GB300.

Workload (the full-size elastic-wall configuration): synthetic aorta-like
vessel on a 128 x 128 x 1024 D3Q19 lattice (tau = 0.8, radius 40 -> 24 along
a seeded spline centreline, two radius-10 side branches), hybrid LV elastance
inlet, three RCR Windkessel outlets, about 2e5 Lagrangian wall nodes with
springs coupled by the penalty immersed boundary; FP32 populations.

One bench step = one time step of the whole hot path: immersed-boundary
interpolation/spreading and wall update, fused stream-collide with bounce-back,
boundary flow/pressure reduction, 0D ODE step and non-equilibrium
extrapolation.  ``value`` = fluid-cell updates per second (MLUPS) over all
ranks, timed with CUDA events on the library's stream (inputs resident in HBM;
the 611 MB population arrays exceed L2, so no flush is needed).  ``e2e`` =
the same through the public API with per-step host I/O: lbm_step_io, whose
step graphs read each step's outlet Windkessel parameters from pinned host
memory and write each step's 0D state rows back to pinned host memory on the
device (with, beside it, the figure for the same I/O as per-step host calls).

``--impl reference`` times the plain FP64 CPU oracle on the same workload
(bounded sample of steps) and prints the same JSON line with impl=reference.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPS & % HBM roofline; time-to-periodic-state vs plain FP32 at 1% error"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76, "f64": 304}
# force density b read by every band cell (three components of the compute type)
BYTES_PER_BAND_CELL = {"f32": 12, "f16": 12, "bf16": 12, "f64": 24}
PROFILE_MD = os.path.join(ROOT, "profiles", "stream_collide_tube_f32.md")
# the sources the stream-collide kernel is compiled from
KERNEL_SRC = [os.path.join(ROOT, "paper_2112_05258_gb300", "csrc", f)
              for f in ("lbm_stream_collide.cu", "lbm_device.cuh")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=24.0)
    ap.add_argument("--workload", choices=["aorta", "batch", "tube"], default="aorta",
                    help="aorta: the full-size elastic-wall case (default); batch: 256 uneven rigid tubes; "
                         "tube: the small 24x24x64 tube the oracle runs in full (latency, not bandwidth)")
    ap.add_argument("--autotune", action="store_true", help="pick block size and occupancy variant first")
    ap.add_argument("--sc-shape", default="", help="BLOCK,VARIANT: fix the stream-collide launch shape (variant 0..4)")
    ap.add_argument("--ib-tpn", type=int, default=0, help="threads per wall node of the node kernel (0: default 4)")
    ap.add_argument("--ib-slabs", type=int, default=0,
                    help="slabs of the pipelined wall-node step (0 or 1: one launch per kernel, the library's default)")
    return ap.parse_args()


def launches(info, steps):
    """Kernel launches of `steps` steps taken as lbm_step does them: whole step
    graphs, then single-step graphs for the rest; a graph's first step (and a
    single step) issues launches_first_step, its later steps launches_per_step."""
    g = info.graph_steps
    full, rest = divmod(steps, g)
    return full * (info.launches_first_step + (g - 1) * info.launches_per_step) + rest * info.launches_first_step


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload(seed, kind="aorta"):
    """Returns (instances, description)."""
    if kind == "batch":
        from workloads import batch
        insts, _ = batch.tube_batch(256, seed)
        desc = (f"batch of 256 rigid tubes, R in [6,20], L in [128,512], LV inlet + RCR outlet each, "
                f"{sum(i.n_fluid for i in insts)} fluid cells, seed {seed}")
        return insts, desc
    if kind == "tube":
        from workloads import configs
        inst = configs.rigid_tube()
        desc = (f"rigid tube {inst.shape[0]}x{inst.shape[1]}x{inst.shape[2]} R=8 tau={inst.tau}, Womersley inlet "
                f"(u_peak 0.02, T 1000) + RCR outlet, {inst.n_fluid} fluid cells (L2-resident)")
        return [inst], desc
    from workloads import aorta
    inst = aorta.build(seed)
    desc = (f"aorta {inst.shape[0]}x{inst.shape[1]}x{inst.shape[2]} tau={inst.tau} LV inlet + 3 RCR outlets, "
            f"{inst.ib.n} IB wall nodes, seed {seed}")
    return [inst], desc


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha256() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def profiled_traffic():
    """dram bytes per stream-collide launch from the committed ncu summary, if
    that summary was taken on the current kernel source (else None)."""
    if not os.path.exists(PROFILE_MD):
        return None
    txt = open(PROFILE_MD).read()
    m1 = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    m2 = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not (m1 and m2):
        return None
    sha = kernel_source_sha256()
    return float(m2.group(1)) if sha == m1.group(1) else None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        time.sleep(0.4)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The maximum of x over all ranks (replicas: the slowest rank decides)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells: int, steps: int, world: int, ms: float) -> float:
    """Whole-job MLUPS of `world` replicas that each update `cells` cells for
    `steps` steps in `ms` milliseconds (the maximum over ranks)."""
    return cells * steps * world / (ms * 1e-3) / 1e6


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _time_oracle(o, seconds: float):
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            return n, dt


def cpu_baseline(inst, seconds: float):
    """Times the FP64 oracle on one instance, about ``seconds`` on one thread
    and as long again on all host cores (the oracle's per-cell loops over
    OpenMP threads; the same bits either way).  The headline entry is the
    all-cores figure; the single-thread one sits beside it."""
    import oracle
    o = oracle.Oracle(inst)
    oracle.set_threads(1)
    n1, dt1 = _time_oracle(o, 0.5 * seconds)
    cores = oracle.set_threads(host_cores())
    nn, dtn = _time_oracle(o, 0.5 * seconds)
    oracle.set_threads(1)
    cells = inst.n_fluid
    return {"value": cells * nn / dtn / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{nn} oracle steps (FP64, {cores} threads) of the same workload, continuing "
                      f"{n1} single-thread steps from rest, {dtn:.1f} s",
            "single_thread": {"value": cells * n1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} oracle steps from rest, {dt1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    insts, desc = workload(args.seed, args.workload)
    inst = insts[0]
    import oracle
    o = oracle.Oracle(inst)
    cores = oracle.set_threads(host_cores())
    budget = 90.0
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    w = min(args.warmup, max(0, int(0.2 * budget / per)))
    if w > 0:
        o.step(w)
    k = max(1, min(args.steps, int(0.8 * budget / per)))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    mlups = inst.n_fluid * k / dt / 1e6
    sample = f"{k} of {args.steps} timed steps (after {w + 1} warm-up), FP64 oracle on {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / k * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "fluid_cells": inst.n_fluid, "parallelism": f"cpu, {cores} threads"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2112_05258_gb300 import Lattice

    insts, desc = workload(args.seed, args.workload)
    inst = insts[0]
    stream = torch.cuda.Stream(device=local)
    wave_cap = 16384 if args.workload == "batch" else 0
    lat = Lattice(insts, precision=args.precision, device=local, stream=stream.cuda_stream, wave_capacity=wave_cap,
                  ib_slabs=args.ib_slabs, ib_threads_per_node=args.ib_tpn)
    info = lat.info()
    tuned = None
    if args.sc_shape:
        blk, var = (int(v) for v in args.sc_shape.split(","))
        lat.set_stream_collide_shape(blk, var)
        tuned = {"block": blk, "variant": var}
    if args.autotune:
        tuned = dict(zip(("block", "min_blocks_per_sm", "cells_per_thread"), lat.autotune(iters=10)))
    cells = info.fluid_cells

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()


    # warm-up (also captures the CUDA graphs)
    lat.step(max(3, args.warmup))
    lat.sync()

    # timed region: K steps of the whole path, CUDA events on the library's stream
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    lat.sync()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device=f"cuda:{local}")
    value = replica_throughput(cells, args.steps, world, ms)

    # dominant kernel: stream-collide, each launch bracketed by events on the same stream
    k_steps = min(args.steps, 400)
    lat.set_kernel_timing(True)
    lat.step(k_steps)
    n_launch, k_ms = lat.kernel_time()
    lat.set_kernel_timing(False)
    per_launch_s = k_ms / n_launch * 1e-3
    # algorithmic bytes of one launch: the populations of every fluid cell,
    # plus the force density at the immersed-boundary band cells
    pop_bytes = BYTES_PER_CELL[args.precision] * cells
    bytes_per_launch = pop_bytes + BYTES_PER_BAND_CELL[args.precision] * info.band_cells
    achieved = bytes_per_launch / per_launch_s / 1e9
    peak, peak_src = measured_peaks()
    traffic = profiled_traffic() if (args.precision == "f32" and args.workload == "aorta") else None

    # end to end through the public API (lbm_step_io): every step the device
    # reads that step's outlet Windkessel parameters from pinned host memory
    # (H2D) and writes the 0D state of all boundaries of the instance into
    # pinned host memory (D2H), in stream order inside the step graphs; the
    # host waits once.  Beside it, the same through per-step host calls
    # (lbm_set_0d_params, lbm_step(h, 1), lbm_read_0d_state_async).
    rcr = np.array(inst.boundaries[1].params, dtype=np.float64)
    nbc = len(inst.boundaries)
    e2e_steps = min(args.steps, 1000)
    params = torch.from_numpy(np.tile(rcr, (e2e_steps, 1))).pin_memory()
    rows = torch.zeros((e2e_steps, 8 * nbc), dtype=torch.float64, pin_memory=True)
    lat.step_io(0, 1, e2e_steps, params.data_ptr(), rcr.size, rows.data_ptr())  # captures the graphs
    lat.sync()
    barrier()
    t0 = time.perf_counter()
    lat.step_io(0, 1, e2e_steps, params.data_ptr(), rcr.size, rows.data_ptr())
    lat.sync()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device=f"cuda:{local}")
    step_of_rows = rows[:, 0].numpy()
    if not np.array_equal(np.diff(step_of_rows), np.ones(e2e_steps - 1)):
        raise RuntimeError("end-to-end read-back rows are not consecutive steps")
    rows2 = torch.zeros((e2e_steps, 8 * nbc), dtype=torch.float64, pin_memory=True)
    barrier()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        lat.set_0d_params(0, 1, rcr)
        lat.step(1)
        lat.state_0d_async(0, rows2[s].data_ptr())
    lat.sync()
    barrier()
    calls_s = max_over_ranks(time.perf_counter() - t0, world, device=f"cuda:{local}")
    if not np.array_equal(np.diff(rows2[:, 0].numpy()), np.ones(e2e_steps - 1)):
        raise RuntimeError("per-step read-back rows are not consecutive steps")
    e2e = {"value": replica_throughput(cells, e2e_steps, world, e2e_s * 1e3), "unit": "MLUPS",
           "h2d_bytes_per_step": int(rcr.nbytes), "d2h_bytes_per_step": int(8 * 8 * nbc),
           "steps": e2e_steps, "api": "lbm_step_io",
           "per_step_calls": {"value": replica_throughput(cells, e2e_steps, world, calls_s * 1e3), "unit": "MLUPS",
                              "api": "lbm_set_0d_params + lbm_step(h, 1) + lbm_read_0d_state_async"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ("aorta", "tube"):
        cpu = cpu_baseline(inst, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": desc, "fluid_cells": cells, "stored_cells": info.stored_cells,
                           "ib_nodes": info.ib_nodes, "precision": args.precision, "autotuned": tuned,
                           "ib_slabs": info.slabs,
                           "launches_per_step": info.launches_per_step,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": ("inputs L2-resident: a latency figure, not a bandwidth one" if args.workload == "tube"
                                  else "inputs larger than L2 (no flush)")},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                             "kernel": "k_stream_collide", "algorithmic_bytes_per_launch": bytes_per_launch,
                             "bytes_per_fluid_cell": BYTES_PER_CELL[args.precision],
                             "bytes_per_band_cell": BYTES_PER_BAND_CELL[args.precision],
                             "band_cells": info.band_cells,
                             "frac_populations_only": pop_bytes / per_launch_s / 1e9 / peak,
                             "launch_ms": per_launch_s * 1e3, "timed_launches": n_launch},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches(info, args.steps),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
