"""Train the load predictor on propagation loads the simulator records itself.

Training data: datapath+FSM designs of the medium shape (seeds 11-14) and of the large
shape (seeds 21-22), each with its own stimulus and sampled stuck-at faults. For every
fault the simulator reports its propagation load (node evaluations summed over the
cycles it was simulated) under the plain schedule; the label is log(1 + load). Features
come from rtlfs_features. Training runs on the GPU through rtlfs_mlp_train (the
library's forward/backward/Adam kernels), from initial weights drawn here with a fixed
seed. Writes the BF16 weights and a JSON report next to this file.

  python -m paper_2508_16376_gb300.train_predictor [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import synth
from .rtlfs import (Simulator, rtlfs_features, rtlfs_mlp_forward, rtlfs_mlp_get_weights,
                    rtlfs_mlp_set_weights, rtlfs_mlp_train, MLP_PARAMS, SCHED_PLAIN)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "predictor_bf16.npy")
REPORT = os.path.join(HERE, "predictor_report.json")


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (nearest, ties to even) and return the bit patterns."""
    f = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((f + 0x7FFF + ((f >> 16) & 1)) >> 16).astype(np.uint16)


def init_weights(seed: int) -> np.ndarray:
    """He-style initial weights for the 5-64-64-1 layout (biases zero)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(MLP_PARAMS, np.float32)
    w[:320] = rng.normal(0, np.sqrt(2 / 5), 320)
    w[384:4480] = rng.normal(0, np.sqrt(2 / 64), 4096)
    w[4544:4608] = rng.normal(0, np.sqrt(1 / 64), 64)
    return bf16_bits(w)


def collect(kind: str, seed: int, n_faults: int, T: int):
    if kind == "medium":
        d = synth.medium_design(seed)
    else:
        rng = np.random.default_rng(seed + 7919)
        states = [int(x) for x in rng.integers(16, 65, 8)]
        d = synth.gen_datapath_fsm(seed, 200000, 20000, 256, 256, states, 0.3, 64, 64, "large")
    stim = synth.stimulus(d, T, seed + 100, 0.1 if kind == "medium" else 0.0)
    f = synth.sample_faults(d, n_faults, seed + 200)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        res, loads = sim.run(want_load=True, scheduler=SCHED_PLAIN)
        X = rtlfs_features(sim.ctx, 0, n_faults)
    return X, np.log1p(loads[0].astype(np.float64)).astype(np.float32)


def spearman(a: np.ndarray, b: np.ndarray) -> float:
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra * rb).sum() / np.sqrt((ra * ra).sum() * (rb * rb).sum()))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="small data, for a smoke check")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args(argv)
    t0 = time.time()
    plan = [("medium", s, 20000, 10000) for s in (11, 12, 13, 14)] + \
           [("large", s, 20000, 4000) for s in (21, 22)]
    if args.quick:
        plan = [("medium", 11, 4000, 2000), ("medium", 12, 4000, 2000)]
    Xs, ys, src = [], [], []
    for kind, seed, F, T in plan:
        X, y = collect(kind, seed, F, T)
        Xs.append(X)
        ys.append(y)
        src.append(dict(kind=kind, seed=seed, faults=F, cycles=T, mean_label=float(y.mean())))
        print(f"collected {kind} seed {seed}: {F} faults, mean log-load {y.mean():.2f}", flush=True)
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    rng = np.random.default_rng(1234)
    perm = rng.permutation(len(y))
    X, y = X[perm], y[perm]
    n_val = len(y) // 10
    Xv, yv, Xt, yt = X[:n_val], y[:n_val], X[n_val:], y[n_val:]
    with Simulator(0) as sim:
        rtlfs_mlp_set_weights(sim.ctx, init_weights(99))
        loss = rtlfs_mlp_train(sim.ctx, Xt, yt, epochs=args.epochs, batch=512, lr=2e-3)
        w = rtlfs_mlp_get_weights(sim.ctx)
        pv = rtlfs_mlp_forward(sim.ctx, Xv)
    mse = float(np.mean((pv - yv) ** 2))
    var = float(np.var(yv))
    heur = Xv[:, 0] * Xv[:, 4]
    report = dict(sources=src, n_train=int(len(yt)), n_val=int(n_val), epochs=args.epochs,
                  final_train_mse=loss, val_mse=mse, val_r2=1 - mse / var if var else None,
                  val_spearman_mlp=spearman(pv, yv), val_spearman_heuristic=spearman(heur, yv),
                  seconds=time.time() - t0)
    np.save(args.out, w)
    with open(REPORT if args.out == WEIGHTS else args.out + ".json", "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
