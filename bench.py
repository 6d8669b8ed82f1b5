"""Benchmark: fault-cycles/s of a full stuck-at fault-simulation campaign on one GB300.

A step is one pass of the whole hot path through the C-ABI (rtlfs_run): good-machine
trace, load prediction and queue order, light and heavy faulty-machine kernels with output
compare, fault dropping and register latch, results to the host. Workload: the medium
datapath+FSM design (20k nodes, 2k registers, 64 inputs / 64 outputs, 32-state FSM),
10k stimulus cycles with 10% held vectors, 100k sampled stuck-at faults. Unit of work:
W = sum over faults of (first detection cycle + 1, or T if undetected) fault-cycles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--faults stuck|transient|mixed] [--no-drop] [--checkpoint-at C]

Under torchrun each rank simulates its own fault sample of the same design (weak
scaling, no data-path collective); value = all ranks' fault-cycles / max rank time.
`--faults` swaps the fault list for transient faults (SEU on register bits, SET on input,
node and output-port bits at uniform cycles) or a mix of stuck-at, output-port and
transient faults; `--no-drop` keeps every fault to the last cycle (the paper's evaluation
protocol), where the work is faults x cycles; `--checkpoint-at C` also times a campaign
stopped at cycle C, saved, loaded into a fresh context and resumed.
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


FAULT_MODELS = {
    "stuck": "stuck-at campaign",
    "transient": "transient-fault campaign (SEU on register bits, SET on input/node/port bits)",
    "mixed": "mixed campaign (stuck-at, output-port stuck-at, transient)",
}


def workload(rank: int, cycles: int = 0, model: str = "stuck"):
    """The medium workload; `cycles` > 0 keeps only the first that many stimulus cycles
    (a short case of the same design and faults, for profiler captures). `model` picks the
    fault list: stuck-at samples, transient faults, or half stuck-at plus every output-port
    fault plus transient faults."""
    from paper_2508_16376_gb300 import synth
    d = synth.medium_design(WORKLOAD["design_seed"])
    stim = synth.stimulus(d, WORKLOAD["cycles"], WORKLOAD["stim_seed"], WORKLOAD["hold_frac"])
    if cycles:
        stim = stim[:cycles]
    F, seed = WORKLOAD["faults"], WORKLOAD["fault_seed"] + rank
    if model == "transient":
        faults = synth.transient_faults(d, F, WORKLOAD["cycles"], seed)
    elif model == "mixed":
        ports = synth.port_faults(d)
        faults = synth.Faults.concat([synth.sample_faults(d, F // 2, seed), ports,
                                      synth.transient_faults(d, F - F // 2 - len(ports), WORKLOAD["cycles"], seed)])
    else:
        faults = synth.sample_faults(d, F, seed)
    return d, stim, faults


def work_units(det, cyc, T: int, no_drop: bool) -> int:
    """W: fault-cycles simulated -- up to the first detection when detected faults are
    dropped, every cycle of every fault in the no-drop mode."""
    return len(det) * T if no_drop else int(np.where(np.asarray(det) == 1, np.asarray(cyc, np.int64) + 1, T).sum())


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


def oracle_sim(d, stim, faults, cores: int, g, no_drop: bool):
    import oracle
    if no_drop:
        return oracle.fault_sim_ex(d, stim, faults, threads=cores, gout=g, no_drop=True)[:3]
    return oracle.fault_sim(d, stim, faults, threads=cores, gout=g)


def cpu_baseline(d, stim, faults, budget_faults: int = 48, seed: int = 5, no_drop: bool = False):
    """The oracle (serial single-fault simulation, one fault per host thread at a time)
    on a bounded random sample of the workload's faults."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(faults), budget_faults, replace=False))
    sample = faults.take(idx)
    cores = os.cpu_count() or 1
    g = oracle.good_outputs(d, stim)
    t0 = time.perf_counter()
    det, cyc, port = oracle_sim(d, stim, sample, cores, g, no_drop)
    dt = time.perf_counter() - t0
    W = work_units(det, cyc, stim.shape[0], no_drop)
    return {"value": W / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{budget_faults} random faults of the workload (seed {seed}), all "
                      f"{stim.shape[0]} cycles, good run excluded; W={W} fault-cycles in {dt:.2f} s"}


def time_checkpoint(sim, d, stim, faults, run_opts, stop: int, device: int) -> dict:
    """Stop the campaign at cycle `stop`, save its state, load it into a fresh context and
    resume; the resumed results and loads must equal an uninterrupted run's."""
    from paper_2508_16376_gb300.rtlfs import Simulator
    res0, loads0 = sim.run(want_load=True, **run_opts)
    full_ms = sim.stats()["total_ms"]
    t0 = time.perf_counter()
    sim.run(stop_cycle=stop, **run_opts)
    stop_ms = sim.stats()["total_ms"]
    t1 = time.perf_counter()
    blob = sim.checkpoint()
    t2 = time.perf_counter()
    with Simulator(device) as sim2:
        sim2.add(d, stim, faults)
        t3 = time.perf_counter()
        sim2.restore(blob)
        t4 = time.perf_counter()
        res1, loads1 = sim2.run(want_load=True, resume=1, **run_opts)
        resume_ms = sim2.stats()["total_ms"]
        t5 = time.perf_counter()
    same = all(np.array_equal(a, b) for a, b in zip(res0, res1)) and \
        all(np.array_equal(a, b) for a, b in zip(loads0, loads1))
    return {"stop_cycle": stop, "bytes": len(blob), "uninterrupted_ms": full_ms,
            "stopped_run_ms": stop_ms, "stopped_run_wall_ms": 1000 * (t1 - t0),
            "save_ms": 1000 * (t2 - t1), "load_ms": 1000 * (t4 - t3),
            "resumed_run_ms": resume_ms, "resumed_run_wall_ms": 1000 * (t5 - t4),
            "results_equal_uninterrupted": bool(same)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    d, stim, faults = workload(0, args.cycles, args.faults)
    g = oracle.good_outputs(d, stim)
    cores = os.cpu_count() or 1
    per_step = max(cores, 16)
    rng = np.random.default_rng(11)
    total_W, times = 0, []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(faults), per_step, replace=False))
        t0 = time.perf_counter()
        det, cyc, port = oracle_sim(d, stim, faults.take(idx), cores, g, args.no_drop)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            total_W += work_units(det, cyc, stim.shape[0], args.no_drop)
    T = sum(times)
    value = total_W / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(config_of(args, stim), sample_per_step=per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random faults per step, all cycles"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(args, stim, **extra):
    c = dict(WORKLOAD, workload=f"medium datapath+FSM RTL design, {FAULT_MODELS[args.faults]}",
             cycles=int(stim.shape[0]), fault_model=args.faults, no_drop=bool(args.no_drop))
    c.update(extra)
    return c


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
    ap.add_argument("--faults", default="stuck", choices=sorted(FAULT_MODELS),
                    help="fault list: stuck-at samples (default), transient faults, or a mix")
    ap.add_argument("--no-drop", action="store_true",
                    help="keep every fault to the last cycle; W = faults x cycles")
    ap.add_argument("--checkpoint-at", type=int, default=0,
                    help="also time a campaign stopped at this cycle (a multiple of the window), "
                         "saved, loaded into a fresh context and resumed")
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
    d, stim, faults = workload(rank, args.cycles, args.faults)
    T = int(stim.shape[0])
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
    if args.no_drop:
        run_opts["no_drop"] = 1
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
    W = len(faults) * T if args.no_drop else stats[-1]["fault_cycles"]
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
    ex = faults.cycle is not None
    fa = rtlfs.fault_array_ex(faults) if ex else rtlfs.fault_array(faults)
    barrier()
    te = []
    for _ in range(max(1, args.steps)):
        t1 = time.perf_counter()
        rtlfs.rtlfs_set_stimulus(sim.ctx, 0, stim)
        if ex:
            rtlfs.rtlfs_set_faults_ex(sim.ctx, 0, fa)
        else:
            rtlfs.rtlfs_set_faults(sim.ctx, 0, fa)
        sim.run(**run_opts)
        if args.no_drop:
            sim.mismatch_counts(0)
        te.append(time.perf_counter() - t1)
    barrier()
    e2e_s = float(np.mean(te))
    t_e = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
    e2e_value = W_all / float(t_e[0])
    h2d = stim.nbytes + fa.nbytes
    d2h = len(faults) * (4 + 4 + 1 + 8 + (4 if args.no_drop else 0))

    last = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(args, stim, n_faults=len(faults),
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

    if rank == 0 and args.checkpoint_at:
        line["checkpoint"] = time_checkpoint(sim, d, stim, faults, run_opts, args.checkpoint_at, local)
    if rank == 0 and args.no_drop:
        line["plain_gpu_form"] = None   # the plain form drops detected faults
    elif rank == 0 and not args.no_plain:
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
        line["cpu_baseline"] = cpu_baseline(d, stim, faults, no_drop=args.no_drop)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
