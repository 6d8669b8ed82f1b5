"""Oracle results for the full-size campaigns, stored under tests/golden/fullsize/.

The oracle (serial single-fault simulation, the problem's definition in Sec. II-B) takes
hours on the full-size workloads, too long for a test, so this script runs it ahead of
time and stores its per-fault results; the GPU tests compare the library's results with
them element by element. Every stored value comes from `oracle.fault_sim`; the inputs come
from `synth` (seeded generators that evaluate nothing). Nothing here calls the CUDA path.

Which faults are checked:
  medium  the bench's medium campaign (20k nodes, 10k cycles): all 100k faults.
  large   the large design (200k nodes, 20k cycles, 1M sampled faults): a stratified
          subsample -- every sampled fault on an FSM state bit, the faults on the sites
          with the most readers (the widest immediate fan-out), and a uniform remainder.
  batch   the 64-design batch: the same rule per design.
The strata are structural (read from the design's arrays), never taken from a GPU run.

  python tests/golden/fullsize_golden.py {medium,large,batch} [--part K[-L]/N] [--threads T]
                                          [--deadline SECONDS] [--out DIR]
                                          [--uniform N] [--fanout M] [--draw D]

A part K/N takes every N-th selected fault starting at K (a uniform sample of the
selection; K-L/N takes parts K..L); with a deadline the script stops taking new faults when it expires and stores
the ones it finished. The tests read every part file of a workload and check the union.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import os
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIR = os.path.join(HERE, "fullsize")

# Subsample sizes: (uniform, widest-fan-out) faults per design; FSM-bit faults are all taken.
LARGE_PICK = (768, 256)
BATCH_PICK = (160, 48)


def _operands_read(op: np.ndarray) -> np.ndarray:
    """How many of the operands a, b, c each node reads (structure only)."""
    from paper_2508_16376_gb300 import synth as s
    n = np.full(op.shape, 2, np.int64)
    n[op == s.CONST] = 0
    n[np.isin(op, [s.NOT, s.SHL, s.SHR, s.SLICE])] = 1
    n[op == s.MUX2] = 3
    return n


def fanout(d) -> np.ndarray:
    """Readers per net: node operands plus register D inputs plus output ports."""
    k = _operands_read(np.asarray(d.node_op))
    cnt = np.zeros(d.n_net, np.int64)
    for j, arr in enumerate((d.node_a, d.node_b, d.node_c)):
        cnt += np.bincount(np.asarray(arr, np.int64)[k > j], minlength=d.n_net)[:d.n_net]
    cnt += np.bincount(np.asarray(d.reg_d, np.int64), minlength=d.n_net)[:d.n_net]
    cnt += np.bincount(np.asarray(d.outputs, np.int64), minlength=d.n_net)[:d.n_net]
    return cnt


def stratified(d, faults, n_uniform: int, n_fanout: int, seed: int) -> np.ndarray:
    """Sorted fault indices: every fault on an FSM state bit, the n_fanout faults whose
    site has the most readers, and n_uniform drawn uniformly."""
    F = len(faults)
    pick = set(np.nonzero(np.isin(faults.net, d.control_nets))[0].tolist())
    fo = fanout(d)[np.asarray(faults.net, np.int64)]
    pick |= set(np.argsort(-fo, kind="stable")[:n_fanout].tolist())
    rng = np.random.default_rng(seed)
    pick |= set(rng.choice(F, min(n_uniform, F), replace=False).tolist())
    return np.array(sorted(pick), np.int64)


def fingerprint(d, stim, faults) -> str:
    """SHA-256 over the arrays the simulators receive (design, stimulus, fault list)."""
    h = hashlib.sha256()
    for a in (d.input_widths, d.reg_widths, d.reg_d, d.node_op, d.node_w, d.node_a, d.node_b,
              d.node_c, d.node_imm, d.outputs, stim, faults.net, faults.bit, faults.val):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def cases(name: str, pick=None, seed_offset: int = 0):
    """[(design index, design, stimulus, faults, selected fault indices)] for a workload;
    `pick` = (uniform, widest fan-out) overrides the subsample sizes and `seed_offset` draws
    another uniform remainder (results already stored for other draws stay valid)."""
    from paper_2508_16376_gb300 import synth
    if name == "medium":
        d, stim, f = synth.workload("medium")
        return [(0, d, stim, f, np.arange(len(f)))]
    if name == "large":
        d, stim, f = synth.workload("large")
        return [(0, d, stim, f, stratified(d, f, *(pick or LARGE_PICK), seed=41 + seed_offset))]
    if name == "batch":
        return [(i, d, stim, f, stratified(d, f, *(pick or BATCH_PICK), seed=4100 + i + 1000 * seed_offset))
                for i, (d, stim, f) in enumerate(synth.batch_workload())]
    raise ValueError(name)


def load(name: str):
    """Union of the stored part files of a workload: dict design index -> (fingerprint,
    fault indices, detected, cycle, port), each sorted by fault index."""
    out = {}
    for path in sorted(glob.glob(os.path.join(DIR, f"{name}_*.npz"))):
        z = np.load(path, allow_pickle=False)
        for di in np.unique(z["design"]):
            m = z["design"] == di
            fp = str(z["fingerprints"][int(di)])
            cur = out.setdefault(int(di), [fp, [], [], [], []])
            assert cur[0] == fp, f"{path}: design {di} was made from other inputs"
            for k, key in enumerate(("idx", "detected", "cycle", "port")):
                cur[1 + k].append(z[key][m])
    res = {}
    for di, (fp, idx, det, cyc, port) in out.items():
        idx, det, cyc, port = (np.concatenate(x) for x in (idx, det, cyc, port))
        idx, first = np.unique(idx, return_index=True)
        res[di] = (fp, idx, det[first], cyc[first], port[first])
    return res


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["medium", "large", "batch"])
    ap.add_argument("--part", default="0/1")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--deadline", type=float, default=0.0, help="seconds; 0 = none")
    ap.add_argument("--out", default=DIR)
    ap.add_argument("--uniform", type=int, default=0, help="uniform faults per design (0: default)")
    ap.add_argument("--fanout", type=int, default=-1, help="widest-fan-out faults per design (-1: default)")
    ap.add_argument("--draw", type=int, default=0, help="another uniform draw (its seed offset)")
    args = ap.parse_args()
    import oracle
    oracle.build()
    ks, n = args.part.split("/")
    n = int(n)
    lo, _, hi = ks.partition("-")
    parts = list(range(int(lo), int(hi or lo) + 1))
    t_start = time.time()
    todo = []   # (design index, fault indices of one chunk)
    ctx = {}
    stored = load(args.name)   # faults already stored under tests/golden/fullsize are skipped
    default = LARGE_PICK if args.name == "large" else BATCH_PICK
    pick = None
    if args.uniform or args.fanout >= 0:
        pick = (args.uniform or default[0], args.fanout if args.fanout >= 0 else default[1])
    for di, d, stim, f, sel in cases(args.name, pick, args.draw):
        mine = np.sort(np.concatenate([sel[k::n] for k in parts]))
        if di in stored:   # faults an earlier run already stored
            mine = mine[~np.isin(mine, stored[di][1])]
        if not len(mine):
            continue
        g = oracle.good_outputs(d, stim)
        ctx[di] = (d, stim, f, g, fingerprint(d, stim, f))
        chunk = 1 if d.n_net > 100000 else 4
        todo += [(di, mine[i:i + chunk]) for i in range(0, len(mine), chunk)]
    fps = [ctx[i][4] if i in ctx else "" for i in range(max(ctx) + 1)] if ctx else []
    print(f"{args.name} parts {parts} of {n}: {sum(len(c) for _, c in todo)} faults in {len(todo)} "
          f"chunks, good runs {time.time() - t_start:.1f} s", flush=True)
    done = []
    lock = threading.Lock()
    stop = threading.Event()
    t0 = time.time()

    def work(item):
        if stop.is_set() or (args.deadline and time.time() - t_start > args.deadline):
            stop.set()
            return
        di, idx = item
        d, stim, f, g, _ = ctx[di]
        det, cyc, port = oracle.fault_sim(d, stim, f.take(idx), threads=1, gout=g)
        with lock:
            done.append((di, idx, det, cyc, port))
            if len(done) % 200 == 0:
                nf = sum(len(x[1]) for x in done)
                print(f"  {nf} faults, {time.time() - t0:.0f} s", flush=True)

    with ThreadPoolExecutor(max(1, args.threads)) as ex:
        list(ex.map(work, todo))
    if not done:
        print("nothing finished")
        return 1
    design = np.concatenate([np.full(len(x[1]), x[0], np.uint16) for x in done])
    arrs = dict(design=design,
                idx=np.concatenate([x[1] for x in done]).astype(np.uint32),
                detected=np.concatenate([x[2] for x in done]).astype(np.uint8),
                cycle=np.concatenate([x[3] for x in done]).astype(np.int32),
                port=np.concatenate([x[4] for x in done]).astype(np.int32),
                fingerprints=np.array(fps))
    os.makedirs(args.out, exist_ok=True)
    tag = f"p{parts[0]:02d}-{parts[-1]:02d}of{n:02d}"
    path = os.path.join(args.out, f"{args.name}_{tag}.npz")
    if os.path.exists(path):   # a part cut short by its deadline: keep both files
        path = os.path.join(args.out, f"{args.name}_{tag}_{int(time.time())}.npz")
    np.savez_compressed(path, **arrs)
    print(f"wrote {path}: {len(design)} faults in {time.time() - t0:.0f} s "
          f"({'cut by deadline' if stop.is_set() else 'complete'})", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
