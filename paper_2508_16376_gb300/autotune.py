"""Autotuner for the campaign knobs: the cycle-window length (overlapped good-trace, light
and heavy kernels; 0 = one pass over all cycles), the light-lane capacity, the fraction of
faults the scheduler sends to the heavy kernel from cycle 0 (the light/heavy split), and
the CTA sizes of the light kernel (lanes per CTA) and of the heavy kernel (threads per
heavy fault), whether the whole good trace runs before the first faulty window
(good_first) or window by window, overlapped with the faulty kernels, and how coarsely the
scheduler orders the queue (order_classes: fine score order, or a few score classes each
kept in fault-list order).

Every candidate is timed with real campaigns through rtlfs_run on the workload loaded in
the simulator (device-event time of the whole campaign, best of `repeats`). The search is
coordinate descent: starting from BASE, each knob in turn takes the value that times
fastest with the others held at the best so far, for `passes` passes. Results never depend
on the knobs, so tuning changes only time. Winners are cached per size bucket (log2 of
total nets, cycles and faults, and the design count) in a JSON file next to this module.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

from .rtlfs import SCHED_HEURISTIC, SCHED_MLP

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")

BASE = dict(window=256, light_cap=1, heavy_frac=0.0, light_block=128, heavy_block=32, good_first=0,
            order_classes=0)
KNOBS: List[Tuple[str, Sequence]] = [
    ("window", (256, 128, 512, 64, 0)),
    ("light_cap", (1, 2)),
    ("heavy_frac", (0.0, 0.02, 0.05)),
    ("light_block", (128, 64, 256)),
    ("heavy_block", (32, 64)),
    ("good_first", (0, 1)),
    ("order_classes", (0, 8, 1)),
]


def fixed_opts(sim, with_mlp: bool) -> Dict:
    """Options every candidate shares: the scheduler, and graph replay for a batch of
    designs (the whole campaign is one captured launch sequence)."""
    o = dict(scheduler=SCHED_MLP if with_mlp else SCHED_HEURISTIC)
    if len(sim.designs) > 1:
        o["use_graph"] = 1
    return o


def size_bucket(sim) -> str:
    nets = sum(d.n_net for d in sim.designs)
    cycles = max(sim.T) if sim.T else 1
    faults = sum(sim.n_faults)
    b = lambda x: int(math.log2(max(1, x)))
    return f"n{b(nets)}_t{b(cycles)}_f{b(faults)}_d{len(sim.designs)}"


def cache_key(sim, with_mlp: bool) -> str:
    return size_bucket(sim) + ("_mlp" if with_mlp else "")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def cached(sim, with_mlp: bool = False, cache_path: str = CACHE) -> Optional[Dict]:
    """The cached winner for the workload loaded in `sim`, or None."""
    e = _load_cache(cache_path).get(cache_key(sim, with_mlp))
    return dict(e["opts"]) if e else None


def tune(sim, repeats: int = 1, passes: int = 1, cache_path: str = CACHE, use_cache: bool = True,
         with_mlp: bool = False, knobs: Optional[List[Tuple[str, Sequence]]] = None,
         verbose: bool = False) -> Dict:
    """Return the fastest option set found for the campaign loaded in `sim` (a Simulator)."""
    key = cache_key(sim, with_mlp)
    cache = _load_cache(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key]["opts"])
    fixed = fixed_opts(sim, with_mlp)
    timed: Dict[str, float] = {}
    trials = []

    def time_of(opts: Dict) -> float:
        k = json.dumps(opts, sort_keys=True)
        if k not in timed:
            ms = float("inf")
            for _ in range(repeats):
                sim.run(**opts)
                ms = min(ms, sim.stats()["total_ms"])
            timed[k] = ms
            trials.append(dict(opts=opts, ms=ms))
            if verbose:
                print(f"autotune {key}: {opts} -> {ms:.1f} ms", flush=True)
        return timed[k]

    best = dict(BASE, **fixed)
    best_ms = time_of(best)
    for _ in range(passes):
        for name, values in (knobs or KNOBS):
            for v in values:
                cand = dict(best, **{name: v})
                ms = time_of(cand)
                if ms < best_ms:
                    best, best_ms = cand, ms
    if use_cache:
        cache = _load_cache(cache_path)
        cache[key] = dict(opts=best, ms=best_ms, trials=trials)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return dict(best)
