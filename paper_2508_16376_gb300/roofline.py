"""Roofline accounting of the campaign's kernels from the library's own counters.

Algorithmic bytes per unit of work (what the method reads or writes by construction,
counting every access once and assuming no reuse across faults or cycles):

* good-trace kernel, per simulated cycle of a design: every net's good value is written
  once (8 B per net) plus the cycle's input vector read (8 B per input);
* light kernel: per fault-cycle it simulates, the site's good value (8 B, the activation
  check); per node evaluation, the node descriptor (16 B), its net record (16 B), the
  node's good value (8 B) and two operand values (16 B) -- 56 B;
* heavy kernel: per node evaluation the same 56 B plus the stamp reads of the two operands
  (8 B) and the stamp+value write of a kept net (12 B) -- 76 B; per fault-cycle 8 B.

The peak is the measured HBM copy bandwidth (MEASURED_PEAKS.json, burst figure); the
fraction is achieved / peak. These kernels are bound by dependent-load latency per fault
rather than by either roof, which the small fractions show.
"""
from __future__ import annotations

import hashlib
import os
from typing import Optional

LIGHT_BYTES_PER_EVAL = 56
LIGHT_BYTES_PER_FAULT_CYCLE = 8
HEAVY_BYTES_PER_EVAL = 76
HEAVY_BYTES_PER_FAULT_CYCLE = 8
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per window launch of 256 cycles, measured with ncu on the medium
# workload's first 1024 cycles (a full-size launch covers the same window and faults); valid
# only for the kernel source they were measured on, identified by its hash.
MEASURED_TRAFFIC = {"light": 59.78e6, "heavy": 117.21e6, "good_trace": 0.76e6}
MEASURED_SOURCE_SHA256_PREFIX = "48bd56eee94319b8"
KERNEL_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "rtlfs_kernels.cu")


def measured_traffic(window: int) -> Optional[dict]:
    """Per-launch DRAM traffic of the window kernels, or None when the kernel source has
    changed since the capture or the window is not the captured one."""
    if window != 256:
        return None
    try:
        with open(KERNEL_SOURCE, "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    return dict(MEASURED_TRAFFIC) if sha.startswith(MEASURED_SOURCE_SHA256_PREFIX) else None


def kernel_bytes(stats: dict, design, T: int) -> dict:
    good = design.n_net * T * 8 + design.n_in * T * 8
    light = (stats["light_evals"] * LIGHT_BYTES_PER_EVAL
             + stats["light_fault_cycles"] * LIGHT_BYTES_PER_FAULT_CYCLE)
    heavy = (stats["heavy_evals"] * HEAVY_BYTES_PER_EVAL
             + stats["heavy_fault_cycles"] * HEAVY_BYTES_PER_FAULT_CYCLE)
    return {"good_trace": good, "light": light, "heavy": heavy}


def kernel_ms(stats: dict) -> dict:
    return {"good_trace": stats["good_ms"], "light": stats["light_ms"], "heavy": stats["heavy_ms"]}


def dominant_roofline(stats: dict, peaks: dict, design, T: int, launches: int = 1,
                      traffic: Optional[dict] = None) -> dict:
    """Roofline entry for the kernel with the largest share of the campaign time. `launches`
    = launches of each window kernel per campaign; achieved = algorithmic bytes per launch /
    average launch duration (the same ratio as the totals); traffic = DRAM bytes per launch."""
    ms = kernel_ms(stats)
    name = max(ms, key=lambda k: ms[k])
    by = kernel_bytes(stats, design, T)
    peak = float(peaks.get("hbm_gbs") or FALLBACK_HBM_GBS)
    n = max(int(launches), 1)
    achieved = (by[name] / n) / (ms[name] / n / 1000.0) / 1e9 if ms[name] > 0 else 0.0
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "algorithmic_bytes_per_launch": int(by[name] / n), "launches": n,
            "avg_launch_ms": ms[name] / n, "traffic": (traffic or {}).get(name)}
