"""Multi-GPU fault sharding: one process per GPU, no data-path collective.

Faults are independent once the design and stimulus are fixed, so a campaign shards over
ranks by fault: every rank loads every design with its whole fault list, predicts the
faults' loads (the library's features and load predictor, or the heuristic cone x toggle
score), takes its share of each list, computes its own good traces and simulates its own
shard; the only exchange is the final gather of per-fault results on the host
(torch.distributed object gather over the process group -- NCCL on GPUs, gloo on CPUs).

Shards are balanced by predicted load with longest-processing-time-first: faults sorted by
descending predicted load go, one by one, to the rank with the smallest total so far. The
predictions are deterministic, so every rank computes the same partition without talking.
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Optional, Sequence

import numpy as np


def lpt_shards(pred_load: np.ndarray, world: int) -> List[np.ndarray]:
    """Fault indices of each rank (each sorted ascending) by longest-processing-time-first."""
    pred = np.asarray(pred_load, np.float64)
    order = np.argsort(-pred, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts: List[list] = [[] for _ in range(world)]
    for i in order:
        tot, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (tot + float(pred[i]), r))
    return [np.sort(np.asarray(p, np.int64)) for p in parts]


def shard_imbalance(pred_load: np.ndarray, shards: Sequence[np.ndarray]) -> float:
    """max over ranks of the predicted load / mean predicted load per rank."""
    tot = np.array([float(np.asarray(pred_load)[s].sum()) for s in shards])
    return float(tot.max() / max(tot.mean(), 1e-30))


def run_sharded(faults, pred_load: np.ndarray, simulate: Callable, group=None):
    """Simulate this rank's shard with simulate(faults_subset) -> (det, cyc, port) and
    gather every rank's results; returns full-length (det, cyc, port) on every rank.
    Without an initialized process group this is the single-process run."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return simulate(faults)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    shards = lpt_shards(pred_load, world)
    mine = shards[rank]
    det, cyc, port = simulate(faults.take(mine))
    gathered: List[Optional[tuple]] = [None] * world
    dist.all_gather_object(gathered, (mine, np.asarray(det), np.asarray(cyc), np.asarray(port)), group=group)
    F = len(faults)
    D = np.zeros(F, np.uint8)
    C = np.full(F, -1, np.int32)
    P = np.full(F, -1, np.int32)
    seen = np.zeros(F, bool)
    for idx, d, c, p in gathered:
        D[idx], C[idx], P[idx] = d, c, p
        seen[idx] = True
    assert seen.all(), "a fault was assigned to no rank"
    return D, C, P


def predicted_loads(sim, use_mlp: bool) -> List[np.ndarray]:
    """Per design of a Simulator, each fault's predicted load: exp of the predictor's log-load
    when `use_mlp` (weights set on the context), else the heuristic score (static cone size
    x toggle rate of the site), both from the library's own kernels."""
    from .rtlfs import rtlfs_features, rtlfs_mlp_forward
    out = []
    for did, n in enumerate(sim.n_faults):
        X = rtlfs_features(sim.ctx, did, n)
        if use_mlp:
            out.append(np.exp(np.minimum(rtlfs_mlp_forward(sim.ctx, X).astype(np.float64), 60.0)))
        else:
            out.append(X[:, 0].astype(np.float64) * X[:, 4] + 1e-9)
    return out


def gather_results(results: Sequence[np.ndarray], mine: Sequence[np.ndarray], sizes: Sequence[int],
                   group=None) -> List[np.ndarray]:
    """Every rank's shard results ([3, n] arrays of detected, cycle, port per design, with
    the fault indices `mine` of each design) gathered into full-length [3, F] arrays."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gathered: List[Optional[tuple]] = [None] * world
    dist.all_gather_object(gathered, [(np.asarray(m), np.asarray(r)) for m, r in zip(mine, results)],
                           group=group)
    full = []
    for di, F in enumerate(sizes):
        out = np.zeros((3, F), np.int64)
        out[1:] = -1
        seen = np.zeros(F, np.int64)
        for per_rank in gathered:
            idx, r = per_rank[di]
            out[:, idx] = r
            seen[idx] += 1
        assert (seen == 1).all(), "the shards are not a partition of the fault list"
        full.append(out)
    return full


def run_sharded_campaign(parts, device: int = 0, run_opts: Optional[dict] = None,
                         weights: Optional[np.ndarray] = None, group=None):
    """One campaign over [(design, stimulus, faults)] split across the process group's ranks
    (one GPU each): every rank predicts the loads, takes its LPT shard of each fault list,
    runs it through rtlfs_run and gathers. Returns full-length [3, F] (detected, cycle,
    port) arrays per design on every rank, and this rank's shards. Without an initialized
    process group this is the single-process campaign."""
    import torch.distributed as dist
    from .rtlfs import Simulator, rtlfs_mlp_set_weights, split
    grouped = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if grouped else 1
    rank = dist.get_rank(group) if grouped else 0
    with Simulator(device) as sim:
        for d, stim, f in parts:
            sim.add(d, stim, f)
        if weights is not None:
            rtlfs_mlp_set_weights(sim.ctx, weights)
        mine = [np.arange(len(f)) for _, _, f in parts]
        if world > 1:
            pred = predicted_loads(sim, use_mlp=weights is not None)
            mine = [lpt_shards(p, world)[rank] for p in pred]
            for did, ((_, _, f), m) in enumerate(zip(parts, mine)):
                sim.set_faults(did, f.take(m))
        res, _ = sim.run(**(run_opts or {}))
    results = [np.stack(split(r)).astype(np.int64) for r in res]
    if world > 1:
        results = gather_results(results, mine, [len(f) for _, _, f in parts], group)
    return results, mine
