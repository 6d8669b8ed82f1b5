"""Multi-GPU fault sharding: one process per GPU, no data-path collective.

Faults are independent once the design and stimulus are fixed, so a campaign shards over
ranks by fault: every rank loads the design, computes its own good trace and simulates its
own shard; the only exchange is the final gather of per-fault results on the host
(torch.distributed object gather over the process group -- NCCL on GPUs, gloo on CPUs).

Shards are balanced by predicted load with longest-processing-time-first: faults sorted by
descending predicted load go, one by one, to the rank with the smallest total so far.
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
