"""Benchmark: fault-cycles/s of a full stuck-at fault-simulation campaign on one GB300.

A step is one pass of the whole hot path through the C-ABI (rtlfs_run): good-machine
trace, load prediction and queue order, light and heavy faulty-machine kernels with output
compare, fault dropping and register latch, results to the host. Workload: the medium
datapath+FSM design (20k nodes, 2k registers, 64 inputs / 64 outputs, 32-state FSM),
10k stimulus cycles with 10% held vectors, 100k sampled stuck-at faults. Unit of work:
W = sum over faults of (first detection cycle + 1, or T if undetected) fault-cycles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank simulates its own fault sample of the same design (weak
scaling, no data-path collective); value = all ranks' fault-cycles / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fault-cycles/sec & campaign wall time vs plain GPU form, bit-exact to oracle"
UNIT = "fault-cycles/s"
WORKLOAD = dict(workload="medium datapath+FSM RTL design, stuck-at campaign",
                nodes=20000, registers=2000, inputs=64, outputs=64, fsm_states=32,
                cycles=10000, hold_frac=0.1, faults=100000, design_seed=2, stim_seed=102,
                fault_seed=202)


# Campaign options the bench times: windows of 256 cycles (good trace, light and heavy
# kernels overlapped on three streams), the small light-lane capacity (4 register diffs,
# 12 net diffs, 12 pending nodes: more faults go to the heavy kernel, whose one-warp form
# handles them cheaply), one warp per heavy fault.
DEFAULT_OPTS = {"window": 256, "light_cap": 1}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(rank: int, cycles: int = 0):
    """The medium workload; `cycles` > 0 keeps only the first that many stimulus cycles
    (a short case of the same design and faults, for profiler captures)."""
    from paper_2508_16376_gb300 import synth
    d = synth.medium_design(WORKLOAD["design_seed"])
    stim = synth.stimulus(d, WORKLOAD["cycles"], WORKLOAD["stim_seed"], WORKLOAD["hold_frac"])
    if cycles:
        stim = stim[:cycles]
    faults = synth.sample_faults(d, WORKLOAD["faults"], WORKLOAD["fault_seed"] + rank)
    return d, stim, faults


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.stop = threading.Event()
        self.th = None

    def __enter__(self):
        def loop():
            while not self.stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.device),
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits"],
                                         capture_output=True, text=True, timeout=5).stdout
                    for line in out.strip().splitlines():
                        self.rows.append([x.strip() for x in line.split(",")])
                except Exception:
                    pass
                self.stop.wait(0.2)
        self.th = threading.Thread(target=loop, daemon=True)
        self.th.start()
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.th:
            self.th.join(timeout=10)
        return False

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def cpu_baseline(d, stim, faults, budget_faults: int = 48, seed: int = 5):
    """The oracle (serial single-fault simulation, one fault per host thread at a time)
    on a bounded random sample of the workload's faults."""
    import oracle
    from paper_2508_16376_gb300 import synth
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(faults), budget_faults, replace=False))
    sample = faults.take(idx)
    cores = os.cpu_count() or 1
    g = oracle.good_outputs(d, stim)
    t0 = time.perf_counter()
    det, cyc, port = oracle.fault_sim(d, stim, sample, threads=cores, gout=g)
    dt = time.perf_counter() - t0
    W = oracle.fault_cycles(det, cyc, stim.shape[0])
    return {"value": W / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{budget_faults} random faults of the workload (seed {seed}), all "
                      f"{stim.shape[0]} cycles, good run excluded; W={W} fault-cycles in {dt:.2f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    d, stim, faults = workload(0, args.cycles)
    g = oracle.good_outputs(d, stim)
    cores = os.cpu_count() or 1
    per_step = max(cores, 16)
    rng = np.random.default_rng(11)
    total_W, times = 0, []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(faults), per_step, replace=False))
        t0 = time.perf_counter()
        det, cyc, port = oracle.fault_sim(d, stim, faults.take(idx), threads=cores, gout=g)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            total_W += oracle.fault_cycles(det, cyc, stim.shape[0])
    T = sum(times)
    value = total_W / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(WORKLOAD, sample_per_step=per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random faults per step, all cycles"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--opts", default=json.dumps(DEFAULT_OPTS),
                    help="rtlfs_run options as JSON (default: the tuned campaign options)")
    ap.add_argument("--cycles", type=int, default=0,
                    help="run only the first N stimulus cycles (a short case for profiling; "
                         "the JSON line names it in config)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16376_gb300 import build as _b
    from paper_2508_16376_gb300 import rtlfs
    from paper_2508_16376_gb300.rtlfs import Simulator
    _b.build()
    d, stim, faults = workload(rank, args.cycles)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    sim = Simulator(local)
    sim.add(d, stim, faults)
    run_opts = json.loads(args.opts)
    # warm-up (also allocates every buffer)
    for _ in range(args.warmup):
        sim.run(**run_opts)
    barrier()
    stats = []
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.run(**run_opts)
            stats.append(sim.stats())
        barrier()
        wall = time.perf_counter() - t0
    dev_ms = [s["total_ms"] for s in stats]
    ms_step = max(float(np.mean(dev_ms)), 1e-9)
    W = stats[-1]["fault_cycles"]
    # max over ranks of the step time, sum of work
    t_rank = torch.tensor([ms_step, float(W)], dtype=torch.float64, device="cuda")
    if dist is not None:
        tmax = t_rank.clone(); dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t_rank.clone(); dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms_all, W_all = float(tmax[0]), float(tsum[1])
    else:
        ms_all, W_all = ms_step, float(W)
    value = W_all / (ms_all / 1000.0)

    # end to end through the ABI with host buffers: stimulus + faults H2D, results D2H
    fa = rtlfs.fault_array(faults)
    barrier()
    te = []
    for _ in range(max(1, args.steps)):
        t1 = time.perf_counter()
        rtlfs.rtlfs_set_stimulus(sim.ctx, 0, stim)
        rtlfs.rtlfs_set_faults(sim.ctx, 0, fa)
        sim.run(**run_opts)
        te.append(time.perf_counter() - t1)
    barrier()
    e2e_s = float(np.mean(te))
    t_e = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
    e2e_value = W_all / float(t_e[0])
    h2d = stim.nbytes + fa.nbytes
    d2h = len(faults) * (4 + 4 + 1 + 8)

    last = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(WORKLOAD, cycles=int(stim.shape[0]),
                           l2="good trace 2 x 8 B x nets x cycles rewritten every step (> L2 at full size)",
                           parallelism=f"fault shards x{ws}", run_opts=run_opts),
            "wall_ms_per_step": 1000 * wall / args.steps,
            "campaign": {k: last[k] for k in ("good_ms", "prep_ms", "light_ms", "heavy_ms",
                                               "promoted", "heavy_initial", "node_evals",
                                               "fault_cycles", "light_evals", "heavy_evals",
                                               "light_fault_cycles", "heavy_fault_cycles")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(last["n_launches"]) * args.steps,
            "clocks": clk.summary()}

    if rank == 0 and not args.no_plain:
        t1 = time.perf_counter()
        sim.run_plain()
        pst = sim.stats()
        line["plain_gpu_form"] = {"value": pst["fault_cycles"] / (pst["total_ms"] / 1000.0),
                                  "unit": UNIT, "ms_per_step": pst["total_ms"],
                                  "wall_s": time.perf_counter() - t1}
    from paper_2508_16376_gb300 import roofline
    window = int(run_opts.get("window", 0))
    n_win = -(-int(stim.shape[0]) // window) if window else 1
    line["roofline"] = roofline.dominant_roofline(last, peaks, d, stim.shape[0], launches=n_win,
                                                  traffic=roofline.measured_traffic(window))
    sim.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(d, stim, faults)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
