"""GPU tests of the sharded campaign driver and the autotuner on small batches: both must
give the oracle's results exactly (neither may change a result, only the time)."""
import os

import numpy as np
import pytest

import oracle
from paper_2508_16376_gb300 import autotune, rtlfs, shard, synth
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _small_batch(n=4):
    out = []
    for i in range(n):
        d = synth.gen_datapath_fsm(60 + i, 1500 + 700 * i, 150 + 70 * i, 16, 16, [8], 0.8, 10, 64, f"s{i}")
        out.append((d, synth.stimulus(d, 300 + 97 * i, 70 + i, 0.1), synth.sample_faults(d, 1500 + 300 * i, 80 + i)))
    return out


def _oracle(parts):
    return [np.stack(oracle.fault_sim(d, s, f, threads=16)).astype(np.int64) for d, s, f in parts]


def test_sharded_campaign_single_rank_equals_oracle():
    parts = _small_batch()
    res, mine = shard.run_sharded_campaign(parts, 0, dict(window=64, light_cap=1, use_graph=1))
    for r, e, m, (_, _, f) in zip(res, _oracle(parts), mine, parts):
        assert np.array_equal(r, e)
        assert np.array_equal(m, np.arange(len(f)))


def test_predicted_loads_and_lpt_shards_partition():
    parts = _small_batch(2)
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        pred = shard.predicted_loads(sim, use_mlp=False)
    for p, (_, _, f) in zip(pred, parts):
        assert p.shape == (len(f),) and np.all(p > 0)
        sh = shard.lpt_shards(p, 3)
        assert np.array_equal(np.sort(np.concatenate(sh)), np.arange(len(f)))
        assert shard.shard_imbalance(p, sh) < 1.1


def test_autotuner_pick_is_oracle_exact(tmp_path):
    parts = _small_batch()
    exp = _oracle(parts)
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        best = autotune.tune(sim, cache_path=str(tmp_path / "cache.json"), verbose=True)
        assert best["use_graph"] == 1
        assert autotune.cached(sim, cache_path=str(tmp_path / "cache.json")) == best
        res, _ = sim.run(**best)
        # and every timed candidate gave the same results: spot-check the extremes of each knob
        for name, values in autotune.KNOBS:
            for v in (values[0], values[-1]):
                r2, _ = sim.run(**dict(best, **{name: v}))
                for a, b in zip(r2, res):
                    assert np.array_equal(a, b), (name, v)
    for r, e in zip(res, exp):
        assert np.array_equal(np.stack(split(r)).astype(np.int64), e)


@pytest.mark.parametrize("window", [64, 256])
def test_good_first_keeps_results(window):
    """The whole good trace before the first faulty window (one launch per design list,
    transposes and activation bitplane over all cycles): the oracle's results, with and
    without graph replay, with and without heavy pre-assignment."""
    parts = _small_batch()
    exp = _oracle(parts)
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        for g, hf in ((0, 0.0), (1, 0.05)):
            res, _ = sim.run(window=window, light_cap=1, good_first=1, use_graph=g, heavy_frac=hf)
            for r, e in zip(res, exp):
                assert np.array_equal(np.stack(split(r)).astype(np.int64), e), (window, g)


@pytest.mark.parametrize("classes", [1, 8, 64])
def test_order_classes_keep_results(classes):
    """The queue ordered by a few score classes, fault-list order kept inside each (with the
    predictor and the heuristic score): the oracle's results."""
    parts = _small_batch()
    exp = _oracle(parts)
    with Simulator(0) as sim:
        for p in parts:
            sim.add(*p)
        rtlfs.rtlfs_mlp_set_weights(sim.ctx, np.load(os.path.join(os.path.dirname(os.path.dirname(
            os.path.abspath(__file__))), "paper_2508_16376_gb300", "predictor_bf16.npy")))
        for sch, hf in ((rtlfs.SCHED_MLP, 0.0), (rtlfs.SCHED_HEURISTIC, 0.05)):
            res, _ = sim.run(window=64, light_cap=1, scheduler=sch, heavy_frac=hf, order_classes=classes)
            for r, e in zip(res, exp):
                assert np.array_equal(np.stack(split(r)).astype(np.int64), e), (classes, sch)
        with pytest.raises(rtlfs.RtlfsError):
            sim.run(window=64, order_classes=3)
