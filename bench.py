"""Benchmark: fault-cycles/s of a full stuck-at fault-simulation campaign on one GB300.

A step is one pass of the whole hot path through the C-ABI, end to end: every design's
stimulus and fault list copied from pinned host memory (rtlfs_set_stimulus,
rtlfs_set_faults), then rtlfs_run -- good-machine trace, features and load prediction,
queue order, light and heavy faulty-machine kernels with output compare, fault dropping
and register latch -- and the per-fault results back in host memory. `value` is the work
over the campaign's device time (CUDA events around its kernels, read from rtlfs_get_stats);
`e2e` is the same work over the step's wall time, copies included.

Unit of work: W = sum over faults of (first detection cycle + 1, or T if undetected)
fault-cycles -- what a simulator that drops each fault at its first detection must do.

Workloads (`--config`):
  learned  (default) the large design (200k nodes, 20k registers, 256/256 ports, 8 FSMs,
           20k cycles, 1M sampled faults) and the 64-design batch (1k-50k nodes, 1k-20k
           cycles, 5k-50k faults each) in one campaign: the trained load predictor orders
           the queue, the windowed campaign is captured into a CUDA graph and replayed;
  large    the large design alone;
  batch    the 64-design batch alone, graph-captured;
  medium   the medium design (20k nodes, 2k registers, 32-state FSM, 10k cycles with 10%
           held vectors, 100k faults); `--faults`, `--no-drop` and `--checkpoint-at` apply here.
Campaign options come from the autotuner's cache (autotune.py) unless `--opts` is given.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--config C]
                  [--faults stuck|transient|mixed] [--no-drop] [--checkpoint-at C]

Under torchrun every rank loads every design and computes the same predicted loads; each
design's fault list is split across ranks by longest-processing-time-first on the predicted
load (shard.py), each rank runs its shards (no data-path collective), and the results are
gathered once after the timed region. value = all ranks' fault-cycles / max rank time.
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

CONFIGS = {
    "learned": dict(workload="large design + 64-design batch in one campaign, learned schedule, "
                             "CUDA-graph replay",
                    designs="large: 200k nodes, 20k regs, 256 in / 256 out, 8 FSMs of 16-64 states, "
                            "20k cycles, 1M sampled stuck-at faults (seeds 4/104/204); batch: 64 "
                            "designs, nodes log-uniform 1k-50k, 1k-20k cycles, 5k-50k faults "
                            "(seeds 1000-1063)",
                    mlp=True),
    "large": dict(workload="large datapath+FSM RTL design, stuck-at campaign",
                  designs="200k nodes, 20k regs, 256 in / 256 out, 8 FSMs of 16-64 states, 20k "
                          "cycles, 1M sampled stuck-at faults (seeds 4/104/204)", mlp=False),
    "batch": dict(workload="64-design batch in one campaign, CUDA-graph replay",
                  designs="64 designs, nodes log-uniform 1k-50k, 1k-20k cycles, 5k-50k faults "
                          "(seeds 1000-1063)", mlp=False),
    "medium": dict(workload="medium datapath+FSM RTL design", designs="20k nodes, 2k regs, "
                   "64 in / 64 out, 32-state FSM, 10k cycles (10% held), 100k faults (seeds "
                   "2/102/202)", mlp=False),
}

# Campaign options used when the autotuner's cache has no entry for the workload (the
# tuner's earlier pick on the medium campaign: windows of 256 cycles, light capacity 1).
DEFAULT_OPTS = {"window": 256, "light_cap": 1}

FAULT_MODELS = {
    "stuck": "stuck-at campaign",
    "transient": "transient-fault campaign (SEU on register bits, SET on input/node/port bits)",
    "mixed": "mixed campaign (stuck-at, output-port stuck-at, transient)",
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(rank: int = 0, cycles: int = 0, model: str = "stuck"):
    """The medium workload; `cycles` > 0 keeps only the first that many stimulus cycles
    (a short case of the same design and faults, for profiler captures). `model` picks the
    fault list: stuck-at samples, transient faults, or half stuck-at plus every output-port
    fault plus transient faults. Every rank gets the same list (ranks shard it)."""
    from paper_2508_16376_gb300 import synth
    d = synth.medium_design(WORKLOAD["design_seed"])
    stim = synth.stimulus(d, WORKLOAD["cycles"], WORKLOAD["stim_seed"], WORKLOAD["hold_frac"])
    if cycles:
        stim = stim[:cycles]
    F, seed = WORKLOAD["faults"], WORKLOAD["fault_seed"]
    if model == "transient":
        faults = synth.transient_faults(d, F, WORKLOAD["cycles"], seed)
    elif model == "mixed":
        ports = synth.port_faults(d)
        faults = synth.Faults.concat([synth.sample_faults(d, F // 2, seed), ports,
                                      synth.transient_faults(d, F - F // 2 - len(ports), WORKLOAD["cycles"], seed)])
    else:
        faults = synth.sample_faults(d, F, seed)
    return d, stim, faults


def parts_of(config: str, cycles: int = 0, model: str = "stuck"):
    """[(design, stimulus, faults)] of a workload; `cycles` > 0 cuts every stimulus."""
    from paper_2508_16376_gb300 import synth
    if config == "medium":
        parts = [workload(0, 0, model)]
    else:
        if model != "stuck":
            raise SystemExit("--faults applies to --config medium only")
        parts = []
        if config in ("learned", "large"):
            parts.append(synth.workload("large"))
        if config in ("learned", "batch"):
            parts += synth.batch_workload()
    if cycles:
        parts = [(d, s[:cycles], f) for d, s, f in parts]
    return parts


def campaign_options(sim, config: str):
    """The options a workload is timed with: the autotuner's cached pick for the workload
    loaded in `sim`, else DEFAULT_OPTS with the options every candidate of the tuner
    shares (scheduler, graph replay for a batch). Returns (options, where they came from)."""
    from paper_2508_16376_gb300 import autotune
    use_mlp = CONFIGS[config]["mlp"]
    o = autotune.cached(sim, with_mlp=use_mlp)
    if o is not None:
        return o, "autotuner cache"
    return dict(DEFAULT_OPTS, **autotune.fixed_opts(sim, use_mlp)), "default (no autotuner entry)"


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


def oracle_sample(parts, n: int, seed: int):
    """n faults drawn uniformly from all the workload's faults (across designs): a list of
    (design index, fault indices)."""
    sizes = np.array([len(f) for _, _, f in parts], np.int64)
    rng = np.random.default_rng(seed)
    flat = np.sort(rng.choice(int(sizes.sum()), min(n, int(sizes.sum())), replace=False))
    first = np.concatenate([[0], np.cumsum(sizes)])
    out = []
    for di in range(len(parts)):
        m = (flat >= first[di]) & (flat < first[di + 1])
        if m.any():
            out.append((di, flat[m] - first[di]))
    return out


def time_oracle(parts, sample, goods, cores: int, no_drop: bool):
    """Wall time and work of the oracle on a sample (one fault per host thread at a time;
    the good runs are computed beforehand and not timed)."""
    t0 = time.perf_counter()
    W = 0
    for di, idx in sample:
        d, stim, f = parts[di]
        det, cyc, port = oracle_sim(d, stim, f.take(idx), cores, goods[di], no_drop)
        W += work_units(det, cyc, stim.shape[0], no_drop)
    return time.perf_counter() - t0, W


def cpu_baseline(parts, n_faults: int = 24, seed: int = 5, no_drop: bool = False):
    """The oracle (serial single-fault simulation) on a bounded random sample of the
    workload's faults, on every host core."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    sample = oracle_sample(parts, n_faults, seed)
    goods = {di: oracle.good_outputs(parts[di][0], parts[di][1]) for di, _ in sample}
    dt, W = time_oracle(parts, sample, goods, cores, no_drop)
    return {"value": W / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sum(len(i) for _, i in sample)} faults drawn uniformly from the workload's "
                      f"fault lists (seed {seed}), all their cycles, good runs excluded; W={W} "
                      f"fault-cycles in {dt:.2f} s"}


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


def config_of(args, parts, **extra):
    c = dict(workload=CONFIGS[args.config]["workload"], config=args.config,
             designs=CONFIGS[args.config]["designs"], n_designs=len(parts),
             nets=int(sum(d.n_net for d, _, _ in parts)),
             cycles_max=int(max(s.shape[0] for _, s, _ in parts)),
             n_faults=int(sum(len(f) for _, _, f in parts)))
    if args.config == "medium":
        c.update(WORKLOAD, workload=f"medium datapath+FSM RTL design, {FAULT_MODELS[args.faults]}",
                 fault_model=args.faults, no_drop=bool(args.no_drop))
    if args.cycles:
        c["cut_to_cycles"] = args.cycles
    c.update(extra)
    return c


def run_reference(args):
    """The oracle on the host cores as the reference arm: each step a bounded sample of the
    workload's faults, timed; rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    parts = parts_of(args.config, args.cycles, args.faults)
    cores = os.cpu_count() or 1
    per_step = max(cores, 16) if args.config == "medium" else cores
    goods = {}
    total_W, times = 0, []
    for s in range(args.warmup + args.steps):
        sample = oracle_sample(parts, per_step, 11 + s)
        for di, _ in sample:
            if di not in goods:
                goods[di] = oracle.good_outputs(parts[di][0], parts[di][1])
        dt, W = time_oracle(parts, sample, goods, cores, args.no_drop)
        if s >= args.warmup:
            times.append(dt)
            total_W += W
    T = sum(times)
    value = total_W / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(args, parts, sample_per_step=per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} faults per step drawn uniformly from the "
                                       f"workload's fault lists, all their cycles, good runs "
                                       f"excluded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _pinned_copy(a: np.ndarray):
    """A copy of `a` in page-locked host memory (torch keeps the allocation alive)."""
    import torch
    t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
    v = t.numpy().view(a.dtype).reshape(a.shape)
    v[...] = a
    return t, v


def plain_comparison(parts, run_opts, device: int, per_design: int, large_cap: int, seed: int = 9):
    """The plain GPU form (one thread per fault, flat launch per design) and the campaign
    with the bench's options on the same subsample: per design min(F, per_design) faults
    (min(F, large_cap) for designs over 100k nets) drawn uniformly."""
    from paper_2508_16376_gb300.rtlfs import Simulator, split
    rng = np.random.default_rng(seed)
    sub = []
    for d, stim, f in parts:
        k = min(len(f), large_cap if d.n_net > 100000 else per_design)
        sub.append((d, stim, f.take(np.sort(rng.choice(len(f), k, replace=False)))))
    with Simulator(device) as sim:
        for d, stim, f in sub:
            sim.add(d, stim, f)
        t0 = time.perf_counter()
        plain = sim.run_plain()
        pst = sim.stats()
        wall = time.perf_counter() - t0
        opts = {k: v for k, v in run_opts.items() if k != "scheduler"}   # no predictor weights here
        ours = sim.run(**opts)[0]
        ost = sim.stats()
    same = all(np.array_equal(np.stack(split(a)), np.stack(split(b))) for a, b in zip(plain, ours))
    return {"value": pst["fault_cycles"] / (pst["total_ms"] / 1000.0), "unit": UNIT,
            "ms": pst["total_ms"], "wall_s": wall,
            "campaign_on_subsample": {"value": ost["fault_cycles"] / (ost["total_ms"] / 1000.0),
                                      "ms": ost["total_ms"]},
            "results_equal": bool(same),
            "subsample": f"{sum(len(f) for _, _, f in sub)} faults: up to {per_design} per design "
                         f"(up to {large_cap} on designs over 100k nets), drawn uniformly (seed {seed})"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="learned", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--opts", default="", help="rtlfs_run options as JSON (default: the autotuner's pick)")
    ap.add_argument("--tune", action="store_true",
                    help="run the autotuner when its cache has no entry for the workload")
    ap.add_argument("--cycles", type=int, default=0,
                    help="run only the first N stimulus cycles (a short case for profiling; "
                         "the JSON line names it in config)")
    ap.add_argument("--faults", default="stuck", choices=sorted(FAULT_MODELS),
                    help="medium only: stuck-at samples (default), transient faults, or a mix")
    ap.add_argument("--no-drop", action="store_true",
                    help="medium only: keep every fault to the last cycle; W = faults x cycles")
    ap.add_argument("--checkpoint-at", type=int, default=0,
                    help="medium only: also time a campaign stopped at this cycle (a multiple of "
                         "the window), saved, loaded into a fresh context and resumed")
    args = ap.parse_args()
    if args.config != "medium" and (args.no_drop or args.checkpoint_at):
        raise SystemExit("--no-drop and --checkpoint-at apply to --config medium only")
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16376_gb300 import autotune, roofline, shard
    from paper_2508_16376_gb300 import build as _b
    from paper_2508_16376_gb300 import rtlfs
    from paper_2508_16376_gb300.rtlfs import Simulator
    _b.build()
    parts = parts_of(args.config, args.cycles, args.faults)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    use_mlp = CONFIGS[args.config]["mlp"]
    weights = np.load(os.path.join(ROOT, "paper_2508_16376_gb300", "predictor_bf16.npy")) if use_mlp else None
    sim = Simulator(local)
    for d, stim, f in parts:
        sim.add(d, stim, f)
    if weights is not None:
        rtlfs.rtlfs_mlp_set_weights(sim.ctx, weights)
    if args.opts:
        run_opts, opts_src = json.loads(args.opts), "--opts"
    elif args.tune and autotune.cached(sim, with_mlp=use_mlp) is None:
        run_opts, opts_src = autotune.tune(sim, with_mlp=use_mlp, verbose=rank == 0), "autotuner"
    else:
        run_opts, opts_src = campaign_options(sim, args.config)
    if args.no_drop:
        run_opts["no_drop"] = 1
    ex = any(f.cycle is not None for _, _, f in parts)

    # Shards: every rank predicts the same loads and takes its LPT share of each list.
    mine = [np.arange(len(f)) for _, _, f in parts]
    if ws > 1:
        pred = shard.predicted_loads(sim, use_mlp=use_mlp)
        mine = [shard.lpt_shards(p, ws)[rank] for p in pred]
    my_parts = [(d, s, f.take(m)) for (d, s, f), m in zip(parts, mine)]
    for did, (_, _, f) in enumerate(my_parts):
        sim.set_faults(did, f)

    # host inputs of every step, page-locked
    pinned = []
    for d, stim, f in my_parts:
        fa = rtlfs.fault_array_ex(f) if ex else rtlfs.fault_array(f)
        pinned.append((_pinned_copy(np.ascontiguousarray(stim, np.uint64)), _pinned_copy(fa)))

    def step():
        t0 = time.perf_counter()
        for did, ((_, sv), (_, fv)) in enumerate(pinned):
            rtlfs.rtlfs_set_stimulus(sim.ctx, did, sv)
            if ex:
                rtlfs.rtlfs_set_faults_ex(sim.ctx, did, fv)
            else:
                rtlfs.rtlfs_set_faults(sim.ctx, did, fv)
        res, _ = sim.run(**run_opts)
        if args.no_drop:
            sim.mismatch_counts(0)
        return time.perf_counter() - t0, res

    for _ in range(args.warmup):
        step()
    barrier()
    stats, walls = [], []
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            w, res = step()
            walls.append(w)
            stats.append(sim.stats())
        barrier()
        wall = time.perf_counter() - t0
    dev_ms = float(np.mean([s["total_ms"] for s in stats]))
    W = sum(len(f) * s.shape[0] for _, s, f in my_parts) if args.no_drop else stats[-1]["fault_cycles"]
    e2e_ms = 1000.0 * float(np.mean(walls))
    t_rank = torch.tensor([dev_ms, e2e_ms, float(W)], dtype=torch.float64, device="cuda")
    if dist is not None:
        tmax = t_rank.clone(); dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t_rank.clone(); dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms_all, e2e_all, W_all = float(tmax[0]), float(tmax[1]), float(tsum[2])
    else:
        ms_all, e2e_all, W_all = dev_ms, e2e_ms, float(W)
    value = W_all / (ms_all / 1000.0)
    h2d = sum(sv.nbytes + fv.nbytes for (_, sv), (_, fv) in pinned)
    d2h = sum(len(f) for _, _, f in my_parts) * (4 + 4 + 1) + (4 * len(my_parts[0][2]) if args.no_drop else 0)

    # results of all ranks gathered once, after the timed region (the only exchange)
    my_results = [np.stack(rtlfs.split(r)).astype(np.int64) for r in res]
    if dist is not None:
        shard.gather_results(my_results, mine, [len(f) for _, _, f in parts])

    last = stats[-1]
    mean = {k: float(np.mean([s[k] for s in stats])) for k in ("good_ms", "light_ms", "heavy_ms")}
    n_win = roofline.windows(run_opts, max(s.shape[0] for _, s, _ in my_parts))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(args, parts,
                                l2="good trace (8 B x nets x cycles, written and read) recomputed "
                                   "every step, far larger than L2",
                                parallelism=f"fault-list shards x{ws} (LPT on predicted load)",
                                run_opts=run_opts, run_opts_source=opts_src),
            "wall_ms_per_step": 1000 * wall / args.steps,
            "campaign": dict({k: last[k] for k in ("promoted", "heavy_initial", "node_evals",
                                                   "fault_cycles", "light_evals", "heavy_evals",
                                                   "light_fault_cycles", "heavy_fault_cycles")},
                             **{k: round(v, 3) for k, v in mean.items()}),
            "e2e": {"value": W_all / (e2e_all / 1000.0), "unit": UNIT, "ms_per_step": e2e_all,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(last["n_launches"]) * args.steps,
            "clocks": clk.summary()}
    ints = roofline.int_peak(peaks, line["clocks"].get("sm_mhz"),
                             torch.cuda.get_device_properties(local).multi_processor_count)
    traffic = (roofline.heavy_traffic_per_launch(last, n_win, last.get("heavy_form") == 3)
               if roofline.dominant(mean)[0] == "heavy" else None)
    line["roofline"] = roofline.step_roofline(my_parts, my_results, last, mean, run_opts,
                                              peaks, n_win, dev_ms, ints, traffic=traffic)
    line["roofline_alu"] = roofline.step_alu(my_parts, last, mean, n_win, dev_ms, ints)
    line["roofline_bound"] = roofline.step_bound(line["roofline"], line["roofline_alu"], dev_ms)

    if rank == 0 and args.checkpoint_at:
        line["checkpoint"] = time_checkpoint(sim, *my_parts[0], run_opts, args.checkpoint_at, local)
    sim.close()
    if rank == 0 and args.no_drop:
        line["plain_gpu_form"] = None   # the plain form drops detected faults
    elif rank == 0 and not args.no_plain:
        full = args.config == "medium"
        line["plain_gpu_form"] = plain_comparison(parts, run_opts, local,
                                                  per_design=100000 if full else 150,
                                                  large_cap=3000)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(parts, 48 if args.config == "medium" else 24,
                                            no_drop=args.no_drop)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
