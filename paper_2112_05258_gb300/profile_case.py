"""Small, self-contained cases for kernel profiling (ncu) and timing sweeps.

    python -m paper_2112_05258_gb300.profile_case --case tube --steps 3
    python -m paper_2112_05258_gb300.profile_case --case aorta --steps 3

``mlp``: the warm-start network (6 -> 256 x 3 -> 64) trained for ``--steps``
Adam steps of 512 samples drawn from 4096 synthetic ones (prints the time
per step).  ``tube``: straight rigid tube, 128 x 128 x 512, radius 40 (2.5M fluid cells,
about 0.4 GB of FP32 populations: larger than L2, small enough for a
multi-pass capture).  ``aorta``: the full-size elastic-wall workload.
``fil_tube``: elastic tube 64 x 64 x 512 whose membrane (radius 24, 151 x 510
nodes) is also 151 axial SGFD filaments; ``spring_tube``: the same membrane
without the filaments.  ``axi``: the axisymmetric straight aorta at 512
nodes per diameter (12802 x 256 = 3.3M nodes, 236 MB of FP32 populations).
Steps are launched directly (no CUDA graph) so that each kernel launch is
visible to a profiler.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="tube",
                    choices=["tube", "aorta", "fil_tube", "spring_tube", "axi", "batch", "mlp"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--nd", type=int, default=512, help="axi: nodes per diameter of the straight aorta")
    ap.add_argument("--warmup", type=int, default=0, help="steps run before the timed ones")
    ap.add_argument("--ib-slabs", type=int, default=1,
                    help="slabs of the pipelined wall-node step (1: one launch per kernel, the profiling default)")
    args = ap.parse_args()
    from paper_2112_05258_gb300 import Lattice
    from workloads import aorta, configs
    if args.case == "mlp":
        import numpy as np
        from paper_2112_05258_gb300.mlp import MLP
        rng = np.random.default_rng(0)
        n_in, n_out, n, batch = 6, 64, 4096, 512
        X = rng.uniform(-1, 1, (n, n_in)).astype(np.float32)
        T = np.tanh(X @ rng.standard_normal((n_in, n_out))).astype(np.float32)
        dims = [n_in, 256, 256, 256, n_out]
        theta = np.concatenate([np.concatenate([rng.standard_normal(dims[k + 1] * dims[k]) / np.sqrt(dims[k]),
                                                np.zeros(dims[k + 1])]) for k in range(4)]).astype(np.float32)
        net = MLP(n_in, 256, 3, n_out, max_batch=n)
        net.set_params(theta)
        net.set_data(X, T)
        order = np.concatenate([rng.permutation(n) for _ in range(args.steps * batch // n + 2)])
        if args.warmup:
            net.train(order[:args.warmup * batch], batch, 1e-3)
        t0 = time.perf_counter()
        losses = net.train(order[:args.steps * batch], batch, 1e-3)
        dt = time.perf_counter() - t0
        print(f"mlp: {args.steps} Adam steps of {batch} in {dt * 1e3:.1f} ms = {dt / args.steps * 1e3:.4f} ms per "
              f"step, loss {losses[0]:.4f} -> {losses[-1]:.5f}")
        net.close()
        return
    if args.case == "axi":
        from paper_2112_05258_gb300.axisym import AxiLattice
        from workloads import axisym
        inst = axisym.straight_aorta(args.nd)
        gs = 64 if args.warmup else 2 * (args.steps + 1)  # timed runs: graphs of 64 steps
        lat = AxiLattice(inst, precision=args.precision, graph_steps=gs)
        if args.warmup:
            lat.step(args.warmup)
            lat.sync()
        t0 = time.perf_counter()
        lat.step(args.steps)
        lat.sync()
        dt = time.perf_counter() - t0
        print(f"axi D/{args.nd} {args.precision}: nodes {inst.node.size} steps {args.steps} in "
              f"{dt * 1e3:.1f} ms = {dt / args.steps * 1e3:.4f} ms per step")
        lat.close()
        return
    insts = None
    if args.case == "batch":
        from workloads import batch
        insts, _ = batch.tube_batch(256, 0)
        inst = insts[0]
    elif args.case == "tube":
        inst = configs.rigid_tube(128, 128, 512, radius=40.0, period=4000)
    elif args.case in ("fil_tube", "spring_tube"):
        inst = configs.ib_tube(64, 64, 512, radius=24.0, period=4000, u_peak=0.02,
                               filaments=args.case == "fil_tube")
    else:
        inst = aorta.build(0)
    lat = Lattice(insts or [inst], precision=args.precision, block_size=args.block,
                  graph_steps=2 * (args.steps + 1),  # graphs longer than the run: single-step graphs only
                  ib_slabs=args.ib_slabs)
    info = lat.info()
    t0 = time.perf_counter()
    lat.step(args.steps)
    lat.sync()
    dt = time.perf_counter() - t0
    print(f"{args.case} {args.precision}: fluid {info.fluid_cells} stored {info.stored_cells} "
          f"ib {info.ib_nodes} steps {args.steps} in {dt * 1e3:.1f} ms")
    lat.close()


if __name__ == "__main__":
    main()
