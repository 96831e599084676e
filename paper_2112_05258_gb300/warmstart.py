"""Learned warm start: predict a periodic-state initialisation from the 0D
parameters, so the coupled solver needs fewer transient beats.

Pipeline (the solver and the network run in the CUDA library; the host only
prepares features and labels and lays out the predicted fields):

1. ``generate``: a batch of tubes with drawn 0D parameters (R_p, C, R_d,
   E_max, E_min, beat period) is run by the batched solver until every
   instance is periodic (cycle-to-cycle waveform change <= 1 %); then, at
   each instance's beat phase 0 (a step that is a multiple of its period),
   its label is read: ventricular and Windkessel-chamber pressures and valve
   state, mean gauge pressure and area-mean velocity of the inlet and outlet
   first fluid layers, and the first 8 radial modes of the axial velocity of
   both layers (Legendre polynomials P_k(2 (r/R)^2 - 1), least squares).
   The 23 values fill the first entries of the 64 network outputs.
2. ``train``: the MLP 6 -> 256 -> 256 -> 256 -> 64 (SiLU) on standardised
   log-features and standardised labels, Adam on the GPU.
3. ``apply``: the predicted label sets the 0D states and an equilibrium
   field (pressure linear along the tube between the two layer pressures,
   axial velocity interpolated linearly between the two mode profiles).

The cold-started method is both the fallback and the reference: warm and cold
runs are compared on the cycles each needs to become periodic and on the
periodic waveforms they reach.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

N_OUT = 64
N_LABEL = 23
N_MODES = 8


def legendre_basis(s: np.ndarray, n: int = N_MODES) -> np.ndarray:
    """P_k(2 s - 1), k < n, for s in [0, 1] (columns)."""
    x = 2.0 * s - 1.0
    out = np.empty((s.size, n))
    out[:, 0] = 1.0
    if n > 1:
        out[:, 1] = x
    for k in range(1, n - 1):
        out[:, k + 1] = ((2 * k + 1) * x * out[:, k] - k * out[:, k - 1]) / (k + 1)
    return out


def features(params: np.ndarray) -> np.ndarray:
    """log R_p, log C, log R_d, E_max, E_min, log T; with 8 columns (the six
    0D parameters, then the tube radius and length) also log R and log L."""
    p = np.asarray(params, dtype=np.float64)
    cols = [np.log(p[:, 0]), np.log(p[:, 1]), np.log(p[:, 2]), p[:, 3], p[:, 4], np.log(p[:, 5])]
    if p.shape[1] >= 8:
        cols += [np.log(p[:, 6]), np.log(p[:, 7])]
    return np.stack(cols, axis=1)


class Layers:
    """Cell indices and radii of an instance's inlet and outlet first layers."""

    def __init__(self, inst):
        nx, ny, nz = inst.shape
        self.shape = (nx, ny, nz)
        self.radius = None
        self.idx, self.s = [], []
        for z in (1, nz - 2):
            yy, xx = np.nonzero(inst.node[z] == 0)
            r2 = (xx + 0.5 - nx / 2) ** 2 + (yy + 0.5 - ny / 2) ** 2
            R2 = (r2.max() + 1e-9) if self.radius is None else self.radius ** 2
            self.radius = np.sqrt(R2) if self.radius is None else self.radius
            self.idx.append(xx + nx * (yy + ny * z))
            self.s.append(r2 / R2)


def read_label(lat, q: int, layers: Layers) -> np.ndarray:
    """The 23 label values of instance q at the current step."""
    P, jx, jy, jz = lat.fields(q)
    lv, rcr = lat.state_0d(q, 0), lat.state_0d(q, 1)
    out = np.zeros(N_OUT)
    out[0], out[1], out[2] = rcr[4], lv[4], lv[6]
    k = 3
    for side in (0, 1):
        idx = layers.idx[side]
        out[k] = P[idx].mean() - 1.0 / 3.0
        out[k + 2] = (jz[idx] / (3.0 * P[idx])).mean()
        k += 1
    k = 7
    for side in (0, 1):
        B = legendre_basis(layers.s[side])
        coef, *_ = np.linalg.lstsq(B, jz[layers.idx[side]], rcond=None)   # velocity v = j / rho0
        out[k:k + N_MODES] = coef
        k += N_MODES
    return out


def apply(lat, q: int, inst, label: np.ndarray, layers: Layers):
    """Sets instance q's state from a (de-standardised) label."""
    nx, ny, nz = layers.shape
    P_in, P_out = label[3], label[4]
    z = np.arange(nz) + 0.5
    frac = np.clip((z - 1.5) / (nz - 3.0), 0.0, 1.0)
    Pz = 1.0 / 3.0 + P_in + (P_out - P_in) * frac
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    s = ((xx - nx / 2) ** 2 + (yy - ny / 2) ** 2).reshape(-1) / layers.radius ** 2
    B = legendre_basis(np.clip(s, 0.0, 1.0))
    u_in = (B @ label[7:7 + N_MODES]) * (s <= 1.0)
    u_out = (B @ label[7 + N_MODES:7 + 2 * N_MODES]) * (s <= 1.0)
    P = np.repeat(Pz, nx * ny)
    uz = (u_in[None, :] * (1 - frac)[:, None] + u_out[None, :] * frac[:, None]).reshape(-1)
    zeros = np.zeros_like(P)
    lat.init_equilibrium(q, P, zeros, zeros, uz)
    valve = 1.0 if label[2] > 0.5 else 0.0
    lat.set_0d_state(q, 0, max(label[1], 0.0), valve_open=valve)
    lat.set_0d_state(q, 1, label[0])


def generate(n: int, seed: int, radius=6.0, length=128, period_range=(2000, 6000), kappa=None,
             precision="f32", max_cycles=20, log=print, geometry_sweep=False, batch_size=256,
             keep_instances=True, radius_range=(6.0, 20.0), length_range=(128, 512)):
    """Runs a sweep to periodic state and reads one label per instance.

    ``geometry_sweep``: radius and length are drawn per instance over
    ``radius_range`` and ``length_range`` (by default the batching workload's
    R in [6, 20], L in [128, 512]) and appended
    to the returned parameters as columns 6 and 7; the sweep runs in batches
    of ``batch_size`` instances (batch b drawn with seed 1000 seed + b).
    Returns (instances or None, params, labels, cycles)."""
    if not geometry_sweep:
        return _generate_batch(n, seed, radius, length, period_range, kappa, precision, max_cycles, log, None)
    insts, params, labels, cycles = [], [], [], []
    for b, k0 in enumerate(range(0, n, batch_size)):
        i, p, y, c = _generate_batch(min(batch_size, n - k0), 1000 * seed + b, radius, length, period_range, kappa,
                                     precision, max_cycles, log, (radius_range, length_range))
        if keep_instances:
            insts += i
        params.append(p)
        labels.append(y)
        cycles.append(c)
    return (insts if keep_instances else None), np.concatenate(params), np.concatenate(labels), \
        np.concatenate(cycles)


def _generate_batch(n, seed, radius, length, period_range, kappa, precision, max_cycles, log, ranges):
    from workloads import batch, configs
    from . import Lattice
    from .periodic import run_to_periodic
    kappa = configs.LV_KAPPA if kappa is None else kappa
    if ranges is not None:
        insts, params, geom = batch.lv_geometry_sweep(n, seed, period_range=period_range, kappa=kappa,
                                                      radius_range=ranges[0], length_range=ranges[1])
        params = np.concatenate([params, geom], axis=1)
    else:
        insts, params = batch.lv_sweep(n, seed, radius=radius, length=length, period_range=period_range,
                                       kappa=kappa)
    periods = params[:, 5].astype(np.int64)
    chunk = 100 if period_range[0] >= 1000 else 20
    cap = int(2 * periods.max() + 2 * chunk)
    lat = Lattice(insts, precision=precision, wave_capacity=cap, graph_steps=chunk)
    t0 = time.perf_counter()
    cycles, steps = run_to_periodic(lat, periods, tol=0.01, max_cycles=max_cycles, chunk=chunk)
    log(f"generate: {n} instances periodic after {steps} steps ({time.perf_counter() - t0:.1f} s); "
        f"cycles median {np.median(cycles):.0f}, unconverged {(cycles < 0).sum()}")
    layers = [Layers(i) for i in insts]
    labels = np.zeros((n, N_OUT))
    pending = np.ones(n, bool)
    while pending.any():
        at0 = pending & (steps % periods == 0)
        for q in np.flatnonzero(at0):
            labels[q] = read_label(lat, q, layers[q])
        pending &= ~at0
        if pending.any():
            lat.step(chunk)
            steps += chunk
    lat.close()
    return insts, params, labels, cycles


def _init_params(shapes, rng):
    return np.concatenate([np.concatenate([rng.standard_normal(r * c) * np.sqrt(1.0 / c), np.zeros(r)])
                           for r, c in shapes]).astype(np.float32)


def layer_shapes(n_in, hidden, n_hidden, n_out):
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[k + 1], dims[k]) for k in range(len(dims) - 1)]


def train(params, labels, hidden=256, n_hidden=3, epochs=300, batch=512, lr=2e-3, seed=0, log=print):
    """Trains the network; returns a predictor (function params -> labels)."""
    from .mlp import MLP
    X = features(params)
    xm, xs = X.mean(0), X.std(0) + 1e-12
    Y = labels[:, :N_LABEL]
    ym, ys = Y.mean(0), Y.std(0) + 1e-12
    Xn = ((X - xm) / xs).astype(np.float32)
    Yn = np.zeros((X.shape[0], N_OUT), np.float32)
    Yn[:, :N_LABEL] = (Y - ym) / ys
    rng = np.random.default_rng(seed)
    batch = max(64, min(batch, (X.shape[0] // 64) * 64))
    n_in = X.shape[1]
    net = MLP(n_in, hidden, n_hidden, N_OUT, max_batch=max(batch, 64))
    net.set_params(_init_params(layer_shapes(n_in, hidden, n_hidden, N_OUT), rng))
    net.set_data(Xn, Yn)
    n = X.shape[0]
    steps_per_epoch = max(1, n // batch)
    order = np.concatenate([rng.permutation(n)[:steps_per_epoch * batch] for _ in range(epochs)])
    t0 = time.perf_counter()
    losses = net.train(order, batch, lr)
    log(f"train: {losses.size} Adam steps in {time.perf_counter() - t0:.1f} s, loss {losses[0]:.4f} -> "
        f"{losses[-50:].mean():.5f}")

    net_batch = max(batch, 64)

    def predict(p):
        Z = ((features(p) - xm) / xs).astype(np.float32)
        nb = ((Z.shape[0] + 63) // 64) * 64
        Zp = np.zeros((nb, Z.shape[1]), np.float32)
        Zp[:Z.shape[0]] = Z
        out = []
        for k in range(0, nb, net_batch):
            out.append(net.forward(Zp[k:k + net_batch]))
        Yp = np.concatenate(out)[:Z.shape[0], :N_LABEL].astype(np.float64) * ys + ym
        full = np.zeros((Z.shape[0], N_OUT))
        full[:, :N_LABEL] = Yp
        return full

    predict.net = net
    predict.losses = losses
    return predict


def evaluate(insts, params, predict, precision_warm="f16", max_cycles=20, log=print, batch_size=None):
    """Cold FP32 start vs warm start (mixed precision, and FP32) on held-out sets.

    ``batch_size``: the held-out instances run in consecutive batches of this
    many (one lattice each, as the batching workload does); wall times add up
    over the batches and the instance that decides each batch is reported."""
    n = len(insts)
    bs = n if not batch_size else int(batch_size)
    parts = [_evaluate_batch(insts[k:k + bs], params[k:k + bs], predict, precision_warm, max_cycles, log)
             for k in range(0, n, bs)]
    res = {}
    for name in parts[0]:
        cyc = np.concatenate([np.array(p[name]["cycles"]) for p in parts])
        ok = cyc >= 0
        r = {"cycles": cyc.tolist(), "steps": [p[name]["steps"] for p in parts],
             "wall_s": float(sum(p[name]["wall_s"] for p in parts)),
             "median_cycles": float(np.median(cyc[ok])) if ok.any() else None,
             "mean_cycles": float(np.mean(cyc[ok])) if ok.any() else None,
             "unconverged": int((~ok).sum()),
             "slowest": [p[name]["slowest"] for p in parts]}
        if "waveform_diffs" in parts[0][name]:
            d = np.concatenate([p[name]["waveform_diffs"] for p in parts])
            r["waveform_diff_vs_cold_max"] = float(d.max())
            r["waveform_diff_vs_cold_median"] = float(np.median(d))
            cc = np.concatenate([np.array(p["cold_f32"]["cycles"]) for p in parts])
            r["fraction_worse_than_cold"] = float(np.mean(cyc > cc))
        res[name] = r
    return res


def _evaluate_batch(insts, params, predict, precision_warm, max_cycles, log):
    from . import Lattice
    from .periodic import run_to_periodic
    periods = params[:, 5].astype(np.int64)
    chunk = 100 if periods.min() >= 1000 else 20
    cap = int(2 * periods.max() + 2 * chunk)
    layers = [Layers(i) for i in insts]
    pred = predict(params)
    res = {}
    finals = {}
    for name, prec, warm in (("cold_f32", "f32", False), ("warm_f32", "f32", True),
                             ("warm_" + precision_warm, precision_warm, True)):
        lat = Lattice(insts, precision=prec, wave_capacity=cap, graph_steps=chunk)
        if warm:
            for q in range(len(insts)):
                apply(lat, q, insts[q], pred[q], layers[q])
        lat.sync()
        t0 = time.perf_counter()
        hist = {}
        cycles, steps = run_to_periodic(lat, periods, tol=0.01, max_cycles=max_cycles, chunk=chunk, history=hist)
        lat.sync()
        wall = time.perf_counter() - t0
        # the instance that decides the batch's wall time: the last to become periodic
        last = int(np.argmax(np.where(cycles >= 0, cycles * periods, int(steps) + 1)))
        # the periodic waveforms reached: the last whole beat (phase 0 to phase 0)
        fin = []
        for q in range(len(insts)):
            T = int(periods[q])
            w = lat.waves(q)
            end = (int(steps) // T) * T
            sel = (w[:, 0] >= end - T) & (w[:, 0] < end)
            fin.append(w[sel, 1:])
        finals[name] = fin
        res[name] = {"cycles": cycles.tolist(), "steps": int(steps), "wall_s": wall,
                     "slowest": {"instance": last, "params": [float(v) for v in params[last]],
                                 "cycles": int(cycles[last]), "cycle_changes": hist.get(last, [])}}
        ok = cycles >= 0
        log(f"{name}: steps {steps}, wall {wall:.2f} s, median cycles "
            f"{float(np.median(cycles[ok])) if ok.any() else None}, unconverged {int((~ok).sum())}")
        lat.close()
    # the periodic state reached from the warm start, against the cold one
    for name in ("warm_f32", "warm_" + precision_warm):
        errs = []
        for q in range(len(insts)):
            a, b = finals[name][q], finals["cold_f32"][q]
            cols = [0, 1, 4, 5]
            errs.append(max(np.abs(a[:, c] - b[:, c]).max() / (np.abs(b[:, c]).max() + 1e-30) for c in cols))
        res[name]["waveform_diffs"] = np.array(errs)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=4096)
    ap.add_argument("--n-test", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--out", default="warmstart.json")
    ap.add_argument("--small", action="store_true", help="short beats and tubes (quick check)")
    ap.add_argument("--geometry-sweep", action="store_true",
                    help="radius and length drawn per instance over the batching workload's ranges")
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    kw = {}
    if a.small:
        from workloads import configs
        kw = dict(radius=4.0, length=32, period_range=(400, 800), kappa=configs.LV_KAPPA * 4000 / 600)
    if a.geometry_sweep:
        kw["geometry_sweep"] = True
    t0 = time.perf_counter()
    _, ptr, ytr, ctr = generate(a.n_train, 1, keep_instances=False, **kw)
    np.savez(os.path.splitext(a.out)[0] + "_train.npz", params=ptr, labels=ytr, cycles=ctr)
    predict = train(ptr, ytr, epochs=a.epochs)
    insts, pte, yte, _ = generate(a.n_test, 2, **kw)
    res = evaluate(insts, pte, predict, batch_size=256 if a.geometry_sweep else None)
    pred = predict(pte)[:, :N_LABEL]
    spread = yte[:, :N_LABEL].std(0)
    err = np.abs(pred - yte[:, :N_LABEL]).mean(0) / np.where(spread > 0, np.abs(yte[:, :N_LABEL]).mean(0), 1.0)
    res["label_rel_err"] = np.where(spread > 0, err, 0.0).tolist()   # constant labels are exact
    res["train_loss_final"] = float(predict.losses[-50:].mean())
    res["total_s"] = time.perf_counter() - t0
    json.dump(res, open(a.out, "w"))
    print(json.dumps({k: v for k, v in res.items() if k not in ("label_rel_err",)}, default=str)[:2000])


if __name__ == "__main__":
    main()
