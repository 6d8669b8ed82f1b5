"""Autotuner for the campaign knobs: cycle windows (overlapped good-trace, light and heavy
kernels) or one pass, light-lane capacity, and the fraction of faults the scheduler sends to
the heavy kernel from cycle 0 (one warp per heavy fault, the heavy form the host picks by
occupancy).

Every candidate is timed with real campaigns through rtlfs_run on the workload loaded in
the simulator (device-event time of the whole campaign, best of `repeats`); the fastest
candidate wins. Results never depend on the knobs, so tuning changes only time. Winners
are cached per size bucket (log2 of total nets, cycles and faults) in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional

from .rtlfs import SCHED_HEURISTIC, SCHED_MLP

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")


def candidates(with_mlp: bool) -> List[Dict]:
    out = []
    sched = SCHED_MLP if with_mlp else SCHED_HEURISTIC
    for window in (256, 0):
        for cap in (1, 2):
            for hf in (0.0, 0.05):
                out.append(dict(scheduler=sched, window=window, light_cap=cap, heavy_frac=hf))
    return out


def size_bucket(sim) -> str:
    nets = sum(d.n_net for d in sim.designs)
    cycles = max(sim.T) if sim.T else 1
    faults = sum(sim.n_faults)
    b = lambda x: int(math.log2(max(1, x)))
    return f"n{b(nets)}_t{b(cycles)}_f{b(faults)}_d{len(sim.designs)}"


def _load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(sim, cands: Optional[List[Dict]] = None, repeats: int = 1, cache_path: str = CACHE,
         use_cache: bool = True, with_mlp: bool = False, verbose: bool = False) -> Dict:
    """Return the fastest option set for the campaign loaded in `sim` (a Simulator)."""
    key = size_bucket(sim) + ("_mlp" if with_mlp else "")
    cache = _load_cache(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key]["opts"])
    cands = cands or candidates(with_mlp)
    best, best_ms, trials = None, float("inf"), []
    for c in cands:
        ms = float("inf")
        for _ in range(repeats):
            sim.run(**c)
            ms = min(ms, sim.stats()["total_ms"])
        trials.append(dict(opts=c, ms=ms))
        if verbose:
            print(f"autotune {key}: {c} -> {ms:.1f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = c, ms
    if use_cache:
        cache[key] = dict(opts=best, ms=best_ms, trials=trials)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return dict(best)
