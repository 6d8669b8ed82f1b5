"""Roofline accounting of a campaign step from its algorithmic counts.

The path has no dense contraction, so the two roofs are HBM bandwidth and the integer
ALU issue rate. Both numerators are algorithmic: what the method must move or compute by
construction, independent of how the kernels happen to do it.

HBM bytes per step:
* the good trace, written once and read once: 2 x 8 B x nets x cycles per design (net
  values are stored as 64-bit words);
* the stimulus read once: 8 B x inputs x cycles;
* the per-fault state carried across cycle-window boundaries: every fault still alive at a
  boundary writes and reads its live-list entry (4 B) and register-diff count (1 B), 10 B
  per crossing (the register-diff entries themselves are not counted: the library's
  counters do not record them);
* the fault descriptors read (8 B) and the results (cycle, port, detected: 9 B) and loads
  (8 B) written once per fault.

Integer operations per step, from the fixed table OPS of 32-bit integer instructions per
op for a result of at most 32 bits / more than 32 bits (a 64-bit value takes two 32-bit
words), plus the width mask (MASK) and, for a faulty evaluation, the compare with the good
value that decides whether the net is kept (KEEP):
* good machine: every node once per cycle, OPS + MASK;
* faulty machines: the recorded node evaluations times the mean of OPS + MASK + KEEP over
  the designs' nodes (the counters record evaluations, not their op mix);
* one output check per simulated fault-cycle.

Peaks: HBM from MEASURED_PEAKS.json (a measured copy); the integer peak is derived as SMs x
INT32 lanes per SM x the SM clock sampled during the timed region, with 128 lanes per SM: a
throughput probe on a GB300 (eight independent add/xor chains per thread, 1216 CTAs of 256
threads) retired 115.8 32-bit integer operations per SM per clock at 2070 MHz, 90% of 128.
"""
from __future__ import annotations

import hashlib
import os
from typing import Dict, List, Optional

import numpy as np

from . import synth as _s

FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of the heavy window kernel (global-bitmap form) from one ncu capture of the
# learned campaign's second window (cycles 256-511 of the large design + 64-design batch,
# windows of 256): read + write bytes of that launch and the heavy evaluations it performed. A launch's traffic is taken
# as proportional to its evaluations; valid while the heavy kernel's source is the captured
# one (the SHA-256 prefix of the text from heavy_run_fault_warp to the light kernel).
HEAVY_CAPTURE = {"dram_bytes": 207.818438e9 + 25.442838e9, "evals": 966_552_453,
                 "source_sha256_prefix": "84d2f8165785c5ea"}
KERNEL_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "rtlfs_kernels.cu")
N_SM = 152
INT32_LANES_PER_SM = 128

OPS = {_s.AND: (1, 2), _s.OR: (1, 2), _s.XOR: (1, 2), _s.NOT: (1, 2), _s.ADD: (1, 2),
       _s.SUB: (1, 2), _s.MUX2: (2, 3), _s.EQ: (1, 2), _s.LT: (1, 2), _s.SHL: (1, 2),
       _s.SHR: (1, 2), _s.SLICE: (1, 2), _s.CONCAT: (2, 4), _s.CONST: (0, 0)}
MASK = (1, 2)
KEEP = (1, 2)
SPILL_BYTES_PER_CROSSING = 10
FAULT_BYTES = 8 + 9 + 8


def heavy_source_sha() -> str:
    try:
        s = open(KERNEL_SOURCE).read()
        a = s.index("template <bool EXACT, bool GBM>\n__device__ __forceinline__ void heavy_run_fault_warp")
        b = s.index("// Light kernel: one lane per fault")
    except (OSError, ValueError):
        return ""
    return hashlib.sha256(s[a:b].encode()).hexdigest()


def heavy_traffic_per_launch(stats: dict, n_win: int, gbm_form: bool) -> Optional[float]:
    """DRAM bytes per heavy launch scaled from the capture by evaluations, or None when the
    kernel changed, the form differs or the capture's evaluation count is not recorded."""
    c = HEAVY_CAPTURE
    if not gbm_form or not c["evals"] or not heavy_source_sha().startswith(c["source_sha256_prefix"]):
        return None
    return c["dram_bytes"] / c["evals"] * stats["heavy_evals"] / max(n_win, 1)


def windows(run_opts: dict, T: int) -> int:
    """Launches of each window kernel per campaign."""
    W = int(run_opts.get("window", 0) or 0)
    return -(-int(T) // W) if W else 1


def node_ops(design) -> tuple:
    """(good-machine ops per cycle, sum over nodes of the faulty evaluation's ops)."""
    op = np.asarray(design.node_op, np.int64)
    wide = (np.asarray(design.node_w, np.int64) > 32).astype(np.int64)
    table = np.array([OPS[k] for k in range(len(OPS))], np.int64)
    base = table[op, wide] + np.array(MASK)[wide]
    return int(base.sum()), int((base + np.array(KEEP)[wide]).sum())


def crossings(parts, results, W: int) -> int:
    """Window boundaries crossed by live faults: sum over faults of ceil(c / W) - 1, c the
    cycles simulated (first detection + 1, or T)."""
    if not W or results is None:
        return 0
    n = 0
    for (d, stim, f), r in zip(parts, results):
        det, cyc = np.asarray(r[0]), np.asarray(r[1], np.int64)
        c = np.where(det == 1, cyc + 1, stim.shape[0])
        n += int(np.sum(np.maximum(-(-c // W) - 1, 0)))
    return n


def step_bytes(parts, results, run_opts: dict) -> Dict[str, int]:
    trace = sum(2 * 8 * d.n_net * s.shape[0] for d, s, _ in parts)
    stim = sum(8 * d.n_in * s.shape[0] for d, s, _ in parts)
    spill = SPILL_BYTES_PER_CROSSING * crossings(parts, results, int(run_opts.get("window", 0) or 0))
    faults = FAULT_BYTES * sum(len(f) for _, _, f in parts)
    return {"good_trace": trace, "stimulus": stim, "window_state": spill, "faults": faults,
            "total": trace + stim + spill + faults}


def step_int_ops(parts, stats: dict) -> Dict[str, int]:
    good = 0
    s_eval, n_nodes = 0, 0
    for d, s, _ in parts:
        g, e = node_ops(d)
        good += g * s.shape[0]
        s_eval += e
        n_nodes += d.n_node
    faulty = int(stats["node_evals"] * (s_eval / max(n_nodes, 1)))
    check = int(stats["fault_cycles"])
    return {"good": good, "faulty": faulty, "output_check": check, "total": good + faulty + check}


def int_peak(peaks: dict, sm_mhz: Optional[float], n_sm: int = N_SM) -> dict:
    mhz = float(sm_mhz or peaks.get("sm_max_mhz") or 2070.0)
    return {"tops": n_sm * INT32_LANES_PER_SM * mhz * 1e6 / 1e12, "n_sm": n_sm,
            "lanes_per_sm": INT32_LANES_PER_SM, "sm_mhz": mhz}


def dominant(mean_ms: dict):
    """The faulty-machine kernel with the larger summed launch time. The good trace is not a
    candidate: in the windowed campaign its figure is the span of its stream, which waits for
    SMs behind the persistent faulty kernels (its kernels' own share of a serialised launch
    list is a few percent)."""
    name = max(("light_ms", "heavy_ms"), key=lambda k: mean_ms[k])
    return {"light_ms": "light", "heavy_ms": "heavy"}[name], mean_ms[name]


def step_roofline(parts, results, stats: dict, mean_ms: dict, run_opts: dict, peaks: dict,
                  n_win: int, step_ms: float, ints: dict, traffic: Optional[float] = None) -> dict:
    """HBM roofline: the step's algorithmic bytes over the dominant kernel's time (its
    launches summed; per launch the same ratio), and over the whole step."""
    by = step_bytes(parts, results, run_opts)
    name, ms = dominant(mean_ms)
    peak = float(peaks.get("hbm_gbs") or FALLBACK_HBM_GBS)
    ach = by["total"] / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
    step = by["total"] / (step_ms / 1000.0) / 1e9 if step_ms > 0 else 0.0
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "algorithmic_bytes_per_step": by["total"], "bytes": by,
            "algorithmic_bytes_per_launch": by["total"] // max(n_win, 1), "launches": n_win,
            "avg_launch_ms": ms / max(n_win, 1), "kernel_ms_per_step": ms,
            "step_achieved": step, "step_frac": step / peak, "traffic": traffic}


def step_bound(hbm: dict, alu: dict, step_ms: float) -> dict:
    """The step's lower bound max(algorithmic bytes / HBM peak, algorithmic integer ops /
    integer peak) and its ratio to the measured step time."""
    t_bytes = hbm["algorithmic_bytes_per_step"] / (hbm["peak"] * 1e9)
    t_ops = alu["int_ops_per_step"] / (alu["peak"] * 1e12)
    bound = max(t_bytes, t_ops)
    return {"bytes_s": t_bytes, "int_ops_s": t_ops, "bound_s": bound,
            "bound_by": "hbm" if t_bytes >= t_ops else "alu", "measured_s": step_ms / 1000.0,
            "frac": bound / (step_ms / 1000.0) if step_ms > 0 else 0.0}


def step_alu(parts, stats: dict, mean_ms: dict, n_win: int, step_ms: float, ints: dict) -> dict:
    """Integer-ALU roofline: the step's algorithmic 32-bit integer operations over the
    dominant kernel's time and over the whole step, against SMs x lanes x clock."""
    ops = step_int_ops(parts, stats)
    name, ms = dominant(mean_ms)
    peak = ints["tops"]
    ach = ops["total"] / (ms / 1000.0) / 1e12 if ms > 0 else 0.0
    step = ops["total"] / (step_ms / 1000.0) / 1e12 if step_ms > 0 else 0.0
    return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "Tops/s",
            "frac": ach / peak, "peak_source": f"derived: {ints['n_sm']} SMs x {ints['lanes_per_sm']} "
                                               f"INT32 lanes x {ints['sm_mhz']:.0f} MHz (sampled)",
            "int_ops_per_step": ops["total"], "ops": ops, "launches": n_win,
            "step_achieved": step, "step_frac": step / peak}
