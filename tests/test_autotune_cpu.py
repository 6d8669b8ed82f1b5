"""The knob autotuner's search and caching logic, against a fake campaign timer (the GPU
campaigns themselves are tuned and checked by tests/test_gpu_autotune.py)."""
import json

from paper_2508_16376_gb300 import autotune

KNOB_NAMES = [k for k, _ in autotune.KNOBS]


class FakeSim:
    """The Simulator attributes the tuner reads, and a campaign time per option set:
    `cost(opts)` gives the milliseconds of a run with those options."""

    def __init__(self, cost, n_net=20000, T=10000, F=100000, n_designs=1):
        self.designs = [type("D", (), {"n_net": n_net})() for _ in range(n_designs)]
        self.T = [T] * n_designs
        self.n_faults = [F] * n_designs
        self.cost = cost
        self.runs = []
        self.last = None

    def run(self, **opts):
        self.runs.append(dict(opts))
        self.last = opts

    def stats(self):
        return {"total_ms": self.cost(self.last)}


def separable(best):
    """A cost whose minimum is `best`, each knob contributing on its own."""
    def cost(o):
        return 1000.0 + sum(10.0 * (o[k] != best[k]) for k in best)
    return cost


def test_knobs_cover_window_split_and_cta_sizes():
    names = dict(autotune.KNOBS)
    assert set(names) == {"window", "light_cap", "heavy_frac", "light_block", "heavy_block", "good_first", "order_classes"}
    assert {64, 128, 256, 512, 0} <= set(names["window"])
    assert len(names["light_block"]) >= 3 and len(names["heavy_block"]) >= 2
    for k, vals in autotune.KNOBS:
        assert autotune.BASE[k] in vals


def test_coordinate_descent_finds_separable_optimum(tmp_path):
    cache = str(tmp_path / "cache.json")
    target = dict(window=128, light_cap=2, heavy_frac=0.05, light_block=64, heavy_block=64, good_first=1, order_classes=8)
    sim = FakeSim(separable(target))
    best = autotune.tune(sim, cache_path=cache)
    assert {k: best[k] for k in target} == target
    assert best["scheduler"] == autotune.SCHED_HEURISTIC and "use_graph" not in best
    # every distinct candidate timed once: the base plus each other value of each knob
    n_distinct = 1 + sum(len(v) - 1 for _, v in autotune.KNOBS)
    assert len(sim.runs) == n_distinct
    data = json.load(open(cache))
    key = autotune.cache_key(sim, False)
    assert data[key]["ms"] == 1000.0 and len(data[key]["trials"]) == n_distinct
    # the same size bucket reuses the cached winner without running
    sim2 = FakeSim(separable(target), n_net=20001)
    assert autotune.cached(sim2, cache_path=cache) == best
    assert autotune.tune(sim2, cache_path=cache) == best and sim2.runs == []
    # the learned schedule is another cache entry
    assert autotune.cached(sim2, with_mlp=True, cache_path=cache) is None


def test_batches_are_tuned_with_graph_replay(tmp_path):
    sim = FakeSim(separable(autotune.BASE), n_designs=64, n_net=12000)
    best = autotune.tune(sim, cache_path=str(tmp_path / "c.json"), with_mlp=True)
    assert best["use_graph"] == 1 and best["scheduler"] == autotune.SCHED_MLP
    assert all(r["use_graph"] == 1 and r["scheduler"] == autotune.SCHED_MLP for r in sim.runs)


def test_repeats_take_the_best_time(tmp_path):
    seq = iter([5.0, 1.0] + [100.0] * 100)
    sim = FakeSim(lambda o: next(seq))
    autotune.tune(sim, cache_path=str(tmp_path / "c.json"), repeats=2)
    data = json.load(open(str(tmp_path / "c.json")))
    assert data[autotune.cache_key(sim, False)]["ms"] == 1.0


def test_cache_off_and_unreadable_cache(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    target = dict(autotune.BASE, window=512)
    sim = FakeSim(separable(target))
    assert autotune.tune(sim, cache_path=str(bad))["window"] == 512
    sim2 = FakeSim(separable(target))
    autotune.tune(sim2, cache_path=str(tmp_path / "none.json"), use_cache=False)
    assert not (tmp_path / "none.json").exists()
