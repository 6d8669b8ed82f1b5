"""The benchmark's contract on the CPU: the reference arm (the oracle on the host cores)
prints one JSON line with the keys the driver reads, the workloads and fault lists are
what the help says, and every rank of a multi-GPU run shards one and the same list."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
from paper_2508_16376_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _reference_line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", *extra],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in KEYS:
        assert k in j, k
    assert j["impl"] == "reference" and j["value"] > 0 and j["unit"] == bench.UNIT
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["cpu_baseline"]["kind"] == "oracle"
    return j


def test_reference_arm_json_line_medium():
    j = _reference_line("--config", "medium", "--cycles", "60", "--faults", "mixed", "--no-drop")
    assert j["config"]["fault_model"] == "mixed" and j["config"]["no_drop"] is True
    assert j["config"]["cut_to_cycles"] == 60


def test_reference_arm_json_line_batch():
    j = _reference_line("--config", "batch", "--cycles", "40")
    assert j["config"]["n_designs"] == 64 and j["config"]["config"] == "batch"


def test_default_workload_is_the_learned_campaign():
    import argparse
    assert bench.CONFIGS["learned"]["mlp"] and "large" in bench.CONFIGS["learned"]["designs"]
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--config", default="learned"' in src


def test_fault_lists_of_the_modes():
    from paper_2508_16376_gb300 import synth
    d, stim, stuck = bench.workload(0, 50)
    assert stim.shape[0] == 50 and len(stuck) == bench.WORKLOAD["faults"] and stuck.cycle is None
    _, _, tr = bench.workload(0, 50, "transient")
    assert len(tr) == bench.WORKLOAD["faults"] and set(np.unique(tr.val)) <= {2, 3}
    _, _, mixed = bench.workload(0, 50, "mixed")
    ports = synth.port_faults(d)
    assert len(mixed) == bench.WORKLOAD["faults"]
    assert np.sum(mixed.net >= d.n_net) >= len(ports)            # every port fault is in
    assert np.sum(mixed.val <= 1) >= bench.WORKLOAD["faults"] // 2 + len(ports)
    # every rank builds the same list: ranks shard it instead of drawing their own
    _, _, other = bench.workload(1, 50)
    assert np.array_equal(other.net, stuck.net)


@pytest.mark.parametrize("world", [2, 4])
def test_rank_shards_partition_one_list(world):
    """What bench.py does per rank under torchrun: every rank computes the same LPT shards
    of each design's list from the same predicted loads and takes its own; the shards of
    all ranks are a partition of the list."""
    rng = np.random.default_rng(world)
    pred = [np.exp(rng.normal(0, 2, n)) for n in (5000, 1234, 7)]
    per_rank = [[shard.lpt_shards(p, world)[r] for p in pred] for r in range(world)]
    for di, p in enumerate(pred):
        allidx = np.sort(np.concatenate([per_rank[r][di] for r in range(world)]))
        assert np.array_equal(allidx, np.arange(len(p)))


def test_work_units():
    det = np.array([1, 0, 1], np.uint8)
    cyc = np.array([4, -1, 0], np.int32)
    assert bench.work_units(det, cyc, 10, False) == 5 + 10 + 1
    assert bench.work_units(det, cyc, 10, True) == 30
