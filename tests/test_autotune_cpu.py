"""The knob autotuner's selection and caching logic, against a fake campaign timer (the
GPU campaigns themselves are timed by the benchmark)."""
import json

from paper_2508_16376_gb300 import autotune


class FakeSim:
    """The Simulator attributes the tuner reads, and a campaign time per option set."""

    def __init__(self, times, n_net=20000, T=10000, F=100000):
        self.designs = [type("D", (), {"n_net": n_net})()]
        self.T = [T]
        self.n_faults = [F]
        self.times = times
        self.runs = []
        self.last = None

    def run(self, **opts):
        self.runs.append(dict(opts))
        self.last = opts

    def stats(self):
        key = (self.last["window"], self.last["light_cap"], self.last["heavy_frac"])
        return {"total_ms": self.times.get(key, 5000.0)}


def test_candidates_cover_the_knobs():
    c = autotune.candidates(False)
    assert len(c) == 8 and len({json.dumps(x, sort_keys=True) for x in c}) == 8
    assert {x["window"] for x in c} == {0, 256} and {x["light_cap"] for x in c} == {1, 2}
    assert all(x["scheduler"] == autotune.SCHED_HEURISTIC for x in c)
    assert all(x["scheduler"] == autotune.SCHED_MLP for x in autotune.candidates(True))


def test_fastest_candidate_wins_and_is_cached(tmp_path):
    cache = str(tmp_path / "cache.json")
    sim = FakeSim({(256, 1, 0.0): 1085.0, (256, 2, 0.0): 1200.0, (0, 1, 0.05): 1900.0})
    best = autotune.tune(sim, cache_path=cache, repeats=2)
    assert (best["window"], best["light_cap"], best["heavy_frac"]) == (256, 1, 0.0)
    assert len(sim.runs) == 16                     # every candidate, twice
    data = json.load(open(cache))
    key = autotune.size_bucket(sim)
    assert data[key]["ms"] == 1085.0 and len(data[key]["trials"]) == 8
    # the same size bucket reuses the cached winner without running
    sim2 = FakeSim({}, n_net=20001)
    assert autotune.tune(sim2, cache_path=cache) == best and sim2.runs == []
    # another bucket, and the learned schedule, are tuned afresh
    sim3 = FakeSim({(0, 2, 0.05): 10.0}, n_net=200000)
    b3 = autotune.tune(sim3, cache_path=cache)
    assert (b3["window"], b3["light_cap"], b3["heavy_frac"]) == (0, 2, 0.05) and len(sim3.runs) == 8
    sim4 = FakeSim({(256, 1, 0.0): 1.0})
    assert autotune.tune(sim4, cache_path=cache, with_mlp=True)["scheduler"] == autotune.SCHED_MLP
    assert len(sim4.runs) == 8


def test_cache_off_and_unreadable_cache(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    sim = FakeSim({(256, 2, 0.05): 3.0})
    best = autotune.tune(sim, cache_path=str(bad))
    assert (best["window"], best["light_cap"], best["heavy_frac"]) == (256, 2, 0.05)
    sim2 = FakeSim({(256, 2, 0.05): 3.0})
    autotune.tune(sim2, cache_path=str(tmp_path / "none.json"), use_cache=False)
    assert not (tmp_path / "none.json").exists()
