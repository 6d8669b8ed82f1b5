"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (its own
workload and options, imported from it), for each fault list and mode it can time.

Every fault is compared with the plain GPU form (one thread per fault, its own kernel and
its own per-thread state). The plain form is not independent of the path under test: it
shares the host's design build (levelizing, renumbering, fan-out and latch maps), the op
evaluator and the good trace, so a mistake there would pass this comparison. What pins the
results to the problem's definition is the oracle: here a stratified sample fault by fault
(the highest propagation loads, the latest detections, faults on FSM state bits and a
uniform remainder), and the stored whole-list oracle results in tests/test_gpu_golden.py.
The load predictor's effect is measured on the medium campaign: identical results, and
whether its ranking of fault loads beats the heuristic's.
"""
import os

import numpy as np
import pytest

import bench
import oracle
from paper_2508_16376_gb300 import rtlfs, synth
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(os.path.dirname(HERE), "paper_2508_16376_gb300", "predictor_bf16.npy")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _stratified(res, loads, faults, design, k, seed):
    det, cyc, _ = split(res)
    rng = np.random.default_rng(seed)
    pick = set(np.argsort(-loads.astype(np.float64))[:k].tolist())
    detected = np.nonzero(det == 1)[0]
    pick |= set(detected[np.argsort(-cyc[detected])[:k]].tolist())
    ctrl = np.nonzero(np.isin(faults.net, design.control_nets))[0]
    if len(ctrl):
        pick |= set(rng.choice(ctrl, min(k, len(ctrl)), replace=False).tolist())
    pick |= set(rng.choice(len(faults), k, replace=False).tolist())
    return np.array(sorted(pick))


def test_medium_full_size():
    """The bench's medium workload (20k nodes, 10k cycles, 100k faults) in the launch
    configuration the bench times it with and in the one-pass form."""
    d, stim, f = bench.workload(0)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        opts, _ = bench.campaign_options(sim, "medium")
        res, loads = sim.run(want_load=True, **opts)
        res1, loads1 = sim.run(want_load=True)
        plain = sim.run_plain()
    for a, b, c in zip(split(res[0]), split(plain[0]), split(res1[0])):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.array_equal(loads[0], loads1[0])
    idx = _stratified(res[0], loads[0], f, d, 12, 1)
    exp = oracle.fault_sim(d, stim, f.take(idx), threads=os.cpu_count() or 4)
    for a, b in zip(split(res[0][idx]), exp):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("model", ["transient", "mixed"])
def test_medium_full_size_fault_models(model):
    """The bench's other fault lists at full size (100k transient faults; stuck-at plus every
    output-port fault plus transient faults): every fault against the plain GPU form, a
    stratified sample against the oracle."""
    d, stim, f = bench.workload(0, 0, model)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        opts, _ = bench.campaign_options(sim, "medium")
        res, loads = sim.run(want_load=True, **opts)
        plain = sim.run_plain()
    for a, b in zip(split(res[0]), split(plain[0])):
        assert np.array_equal(a, b)
    idx = _stratified(res[0], loads[0], f, d, 8, 3)
    exp = oracle.fault_sim(d, stim, f.take(idx), threads=os.cpu_count() or 4)
    for a, b in zip(split(res[0][idx]), exp):
        assert np.array_equal(a, b)


def test_medium_full_size_no_drop():
    """The no-drop mode at full size (every fault to the last cycle): first detections and
    mismatch-cycle counts of a stratified sample against the oracle's no-drop run."""
    d, stim, f = bench.workload(0, 0, "mixed")
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        res, loads = sim.run(want_load=True, no_drop=1, **bench.DEFAULT_OPTS)
        cnt = sim.mismatch_counts(0)
    idx = _stratified(res[0], loads[0], f, d, 6, 4)
    exp = oracle.fault_sim_ex(d, stim, f.take(idx), threads=os.cpu_count() or 4, no_drop=True)
    for a, b in zip(split(res[0][idx]), exp[:3]):
        assert np.array_equal(a, b)
    assert np.array_equal(cnt[idx], exp[3])


def test_medium_full_size_checkpoint():
    """A full-size campaign stopped at cycle 5120, saved, loaded into a fresh context and
    resumed equals the uninterrupted campaign (results and loads)."""
    d, stim, f = bench.workload(0)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        ref, ref_loads = sim.run(want_load=True, **bench.DEFAULT_OPTS)
        sim.run(stop_cycle=5120, **bench.DEFAULT_OPTS)
        blob = sim.checkpoint()
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        sim.restore(blob)
        res, loads = sim.run(want_load=True, resume=1, **bench.DEFAULT_OPTS)
    assert np.array_equal(res[0], ref[0])
    assert np.array_equal(loads[0], ref_loads[0])


def test_large_design_subsample():
    """200k nodes, 20k registers, 256/256 ports, 8 FSMs, all 20k cycles; 3000 of the
    sampled faults (one wave of the plain form) in the large campaign's benchmark options,
    every one against the plain GPU form; a stratified handful against the oracle."""
    d = synth.large_design(4)
    stim = synth.stimulus(d, 20000, 104)
    f = synth.sample_faults(d, 3000, 204)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        opts, _ = bench.campaign_options(sim, "large")
        res, loads = sim.run(want_load=True, **opts)
        res2 = sim.run_plain()
    for a, b in zip(split(res[0]), split(res2[0])):
        assert np.array_equal(a, b)
    idx = _stratified(res[0], loads[0], f, d, 3, 2)
    exp = oracle.fault_sim(d, stim, f.take(idx), threads=os.cpu_count() or 4)
    for a, b in zip(split(res[0][idx]), exp):
        assert np.array_equal(a, b)


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra * rb).sum() / np.sqrt((ra * ra).sum() * (rb * rb).sum()))


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained predictor weights")
def test_learned_scheduler_gain():
    """Trained predictor vs the heuristic on a medium campaign the predictor never saw
    (fault seed 303): results identical; the predictor ranks the recorded loads better
    than the static-cone x toggle-rate heuristic; the campaign times are reported."""
    d = synth.medium_design(2)
    stim = synth.stimulus(d, 10000, 102, 0.1)
    f = synth.sample_faults(d, 100000, 303)
    w = np.load(WEIGHTS)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        rtlfs.rtlfs_mlp_set_weights(sim.ctx, w)
        X = rtlfs.rtlfs_features(sim.ctx, 0, len(f))
        pred = rtlfs.rtlfs_mlp_forward(sim.ctx, X)
        times = {}
        ref = None
        for name, kw in [("plain", dict(scheduler=rtlfs.SCHED_PLAIN)),
                         ("heuristic", dict(scheduler=rtlfs.SCHED_HEURISTIC, heavy_frac=0.05)),
                         ("mlp", dict(scheduler=rtlfs.SCHED_MLP, heavy_frac=0.05))]:
            res, loads = sim.run(want_load=True, **kw)
            times[name] = sim.stats()["total_ms"]
            r = split(res[0])
            if ref is None:
                ref, L = r, loads[0]
            for a, b in zip(r, ref):
                assert np.array_equal(a, b)
    y = np.log1p(L.astype(np.float64))
    s_mlp = _spearman(pred, y)
    s_heur = _spearman(X[:, 0] * X[:, 4], y)
    print(f"campaign ms {times}; rank correlation with load: mlp {s_mlp:.3f} heuristic {s_heur:.3f}")
    assert s_mlp > s_heur
