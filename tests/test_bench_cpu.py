"""The benchmark's contract on the CPU: the reference arm (the oracle on the host cores)
prints one JSON line with the keys the driver reads, and the fault lists and work unit of
the benchmark's modes are what its help says."""
import json
import os
import subprocess
import sys

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cycles", "60", "--faults", "mixed", "--no-drop"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["impl"] == "reference" and j["value"] > 0 and j["unit"] == bench.UNIT
    assert j["config"]["fault_model"] == "mixed" and j["config"]["no_drop"] is True
    assert j["config"]["cycles"] == 60
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["cpu_baseline"]["kind"] == "oracle"


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
    # a second rank samples its own faults of the same design
    _, _, other = bench.workload(1, 50)
    assert not np.array_equal(other.net, stuck.net)


def test_work_units():
    det = np.array([1, 0, 1], np.uint8)
    cyc = np.array([4, -1, 0], np.int32)
    assert bench.work_units(det, cyc, 10, False) == 5 + 10 + 1
    assert bench.work_units(det, cyc, 10, True) == 30
