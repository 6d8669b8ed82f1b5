"""Parity with the oracle at the full sizes of every campaign configuration, in the exact
options the benchmark times each one with.

The oracle's per-fault results were computed ahead of time by tests/golden/
fullsize_golden.py, which runs only the oracle on the synth inputs (the medium campaign's
whole fault list; structural stratified subsamples of the large design and of each of the
64 batch designs: every fault on an FSM state bit, the faults on the sites with the most
readers, and a uniform remainder). Each test runs the whole campaign on the GPU and
compares every stored fault element by element (detected flag, first cycle, first port).
The stored inputs' fingerprints must match the inputs the test builds.
"""
import os
import sys

import numpy as np
import pytest

import bench
from paper_2508_16376_gb300 import rtlfs
from paper_2508_16376_gb300.rtlfs import Simulator, split

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fullsize_golden as golden  # noqa: E402

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(HERE), "paper_2508_16376_gb300", "predictor_bf16.npy")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def large_and_batch():
    return bench.parts_of("large"), bench.parts_of("batch")


def _check(name, parts, results, offset=0):
    """Compare the stored oracle results of workload `name` with the GPU results of its
    designs (results[offset + design index]); returns the number of faults compared."""
    stored = golden.load(name)
    assert stored, f"no stored oracle results for {name}"
    n = 0
    for di, (fp, idx, det, cyc, port) in stored.items():
        d, stim, f = parts[offset + di]
        assert golden.fingerprint(d, stim, f) == fp, f"{name} design {di}: inputs differ from the stored ones"
        gdet, gcyc, gport = (np.asarray(x)[idx] for x in split(results[offset + di]))
        bad = np.nonzero((gdet != det) | (gcyc != cyc) | (gport != port))[0]
        assert len(bad) == 0, (f"{name} design {di}: {len(bad)} of {len(idx)} faults differ from the "
                               f"oracle, first fault {idx[bad[0]]}: gpu {gdet[bad[0]], gcyc[bad[0]], gport[bad[0]]} "
                               f"oracle {det[bad[0]], cyc[bad[0]], port[bad[0]]}")
        n += len(idx)
    return n


def test_medium_all_faults_vs_oracle():
    """The medium campaign (20k nodes, 10k cycles, 100k faults) in the benchmark's options;
    every stored fault of the oracle's whole-list results."""
    parts = bench.parts_of("medium")
    with Simulator(0) as sim:
        sim.add(*parts[0])
        opts, src = bench.campaign_options(sim, "medium")
        res, _ = sim.run(**opts)
    n = _check("medium", parts, res)
    print(f"medium: {n} of {len(parts[0][2])} faults bit-exact to the oracle ({src}: {opts})")


def test_large_subsample_vs_oracle(large_and_batch):
    """The large design's whole campaign (1M faults, 20k cycles) in the benchmark's options
    for it; the stored stratified subsample against the oracle."""
    parts = large_and_batch[0]
    with Simulator(0) as sim:
        sim.add(*parts[0])
        opts, src = bench.campaign_options(sim, "large")
        res, _ = sim.run(**opts)
    n = _check("large", parts, res)
    print(f"large: {n} faults bit-exact to the oracle ({src}: {opts})")


def test_batch_subsamples_vs_oracle(large_and_batch):
    """The 64-design batch in one graph-captured campaign in the benchmark's options for it;
    each design's stored stratified subsample against the oracle."""
    parts = large_and_batch[1]
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        opts, src = bench.campaign_options(sim, "batch")
        assert opts.get("use_graph") == 1
        res, _ = sim.run(**opts)
    n = _check("batch", parts, res)
    print(f"batch: {n} faults over {len(parts)} designs bit-exact to the oracle ({src}: {opts})")


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained predictor weights")
def test_learned_campaign_vs_oracle_and_heuristic(large_and_batch):
    """The learned-scheduled campaign (large design + 64-design batch, one graph-captured
    campaign ordered by the trained predictor) in the benchmark's options: the stored oracle
    results of both workloads, and every fault against the same campaign under the heuristic
    schedule. Prints both campaign times (the predictor's measured gain or loss)."""
    large, batch = large_and_batch
    parts = large + batch
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        rtlfs.rtlfs_mlp_set_weights(sim.ctx, np.load(WEIGHTS))
        opts, src = bench.campaign_options(sim, "learned")
        assert opts["scheduler"] == rtlfs.SCHED_MLP and opts.get("use_graph") == 1
        times = {}
        res, _ = sim.run(**opts)
        res, _ = sim.run(**opts)   # the second replay of the captured graph
        times["mlp"] = sim.stats()["total_ms"]
        heur = dict(opts, scheduler=rtlfs.SCHED_HEURISTIC)
        sim.run(**heur)
        href, _ = sim.run(**heur)
        times["heuristic"] = sim.stats()["total_ms"]
    n = _check("large", parts, res) + _check("batch", parts, res, offset=1)
    for a, b in zip(res, href):
        assert np.array_equal(a, b)
    gain = times["heuristic"] / times["mlp"]
    print(f"learned: {n} faults bit-exact to the oracle, all {sum(len(p[2]) for p in parts)} equal to the "
          f"heuristic schedule; campaign ms {times}, heuristic/mlp = {gain:.3f} ({src}: {opts})")
