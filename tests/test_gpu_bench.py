"""The benchmark's own arm on a GB300, on short cases of two workloads: one JSON line with
the keys the driver reads, both roofline entries reproducible from the line's own counts,
and the plain GPU form and the campaign agreeing on the subsample they are timed on."""
import json
import os
import subprocess
import sys

import pytest

import bench

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "1",
                          "--no-cpu-baseline", *args], capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("config,cycles", [("batch", 300), ("medium", 600)])
def test_bench_line(config, cycles):
    j = _line("--config", config, "--cycles", str(cycles))
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks",
              "roofline", "roofline_alu", "roofline_bound", "plain_gpu_form"):
        assert k in j, k
    assert j["metric"] == bench.METRIC and j["unit"] == bench.UNIT and j["steps"] == 2
    assert j["value"] > 0 and j["e2e"]["value"] > 0 and j["e2e"]["h2d_bytes_per_step"] > 0
    assert j["e2e"]["value"] <= j["value"] * 1.001          # wall time includes the device time
    assert j["gpu_launches"] > 0
    r, a = j["roofline"], j["roofline_alu"]
    assert r["bound"] == "hbm" and a["bound"] == "alu"
    ms = r["kernel_ms_per_step"]
    assert abs(r["achieved"] - r["algorithmic_bytes_per_step"] / (ms / 1000) / 1e9) <= 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-9
    assert abs(a["frac"] - a["achieved"] / a["peak"]) <= 1e-9
    assert a["int_ops_per_step"] == sum(v for k, v in a["ops"].items() if k != "total")
    assert j["plain_gpu_form"]["results_equal"] is True
    if config == "batch":
        assert j["config"]["n_designs"] == 64 and j["config"]["run_opts"].get("use_graph") == 1
