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

from typing import Optional

LIGHT_BYTES_PER_EVAL = 56
LIGHT_BYTES_PER_FAULT_CYCLE = 8
HEAVY_BYTES_PER_EVAL = 76
HEAVY_BYTES_PER_FAULT_CYCLE = 8
FALLBACK_HBM_GBS = 6800.0


def kernel_bytes(stats: dict, design, T: int) -> dict:
    good = design.n_net * T * 8 + design.n_in * T * 8
    light = (stats["light_evals"] * LIGHT_BYTES_PER_EVAL
             + stats["light_fault_cycles"] * LIGHT_BYTES_PER_FAULT_CYCLE)
    heavy = (stats["heavy_evals"] * HEAVY_BYTES_PER_EVAL
             + stats["heavy_fault_cycles"] * HEAVY_BYTES_PER_FAULT_CYCLE)
    return {"good_trace": good, "light": light, "heavy": heavy}


def kernel_ms(stats: dict) -> dict:
    return {"good_trace": stats["good_ms"], "light": stats["light_ms"], "heavy": stats["heavy_ms"]}


def dominant_roofline(stats: dict, peaks: dict, design, T: int,
                      traffic: Optional[dict] = None) -> dict:
    """Roofline entry for the kernel with the largest share of the campaign time."""
    ms = kernel_ms(stats)
    name = max(ms, key=lambda k: ms[k])
    by = kernel_bytes(stats, design, T)
    peak = float(peaks.get("hbm_gbs") or FALLBACK_HBM_GBS)
    achieved = by[name] / (ms[name] / 1000.0) / 1e9 if ms[name] > 0 else 0.0
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "algorithmic_bytes": int(by[name]), "kernel_ms": ms[name],
            "traffic": (traffic or {}).get(name)}
