"""The cluster form of the good trace (one thread-block cluster of 2-16 CTAs per design,
net values in distributed shared memory, register banks by cycle parity): the trace equals
the oracle's net by net and the fault results equal the oracle's, for every cluster size,
levels narrower than the cluster (CTAs with nothing to do at a level), levels wider than one
chunk per CTA, registers fed by registers (the parity banks), window resumption, and the
automatic choice for a design too large for one CTA."""
import functools

import numpy as np
import pytest

import oracle
from paper_2508_16376_gb300 import synth
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _run(d, stim, faults, **opts):
    with Simulator(0) as sim:
        sim.add(d, stim, faults)
        res, _ = sim.run(**opts)
        trace = sim.good_trace(0)
    return split(res[0]), trace


def _big_design():
    # 30k nodes over ~25 levels: wider than one 512-node chunk per CTA at C = 2
    return synth.gen_datapath_fsm(5, 30000, 600, 32, 32, [16], 0.5, 20, 64, "big")


@functools.lru_cache(maxsize=None)
def _case(which):
    """(design, stimulus, faults, oracle trace, oracle results) of a named case."""
    if which == "tiny":   # 200 nodes: most levels narrower than the cluster
        d = synth.tiny_design(1)
        stim = synth.stimulus(d, 100, 101)
        f = synth.fault_universe(d)
    elif which == "fsm":
        d = synth.gen_datapath_fsm(3, 3000, 300, 16, 16, [8], 0.8, 12, 64, "fsm3")
        stim = synth.stimulus(d, 333, 11, 0.1)
        f = synth.sample_faults(d, 1500, 7)
    elif which == "fsm300":
        d = synth.gen_datapath_fsm(3, 3000, 300, 16, 16, [8], 0.8, 12, 64, "fsm3")
        stim = synth.stimulus(d, 300, 12, 0.1)
        f = synth.sample_faults(d, 1200, 8)
    elif which == "chain":
        d = synth.delay_chain(9, 13)
        stim = synth.stimulus(d, 60, 3)
        f = synth.fault_universe(d)
    else:
        d = _big_design()
        stim = synth.stimulus(d, 96, 5)
        f = synth.sample_faults(d, 800, 1)
    _, trace = oracle.good_run(d, stim, with_trace=True)
    exp = oracle.fault_sim(d, stim, f, threads=16)
    return d, stim, f, trace, exp


def _check(which, **opts):
    d, stim, f, trace, exp = _case(which)
    got, gt = _run(d, stim, f, **opts)
    assert np.array_equal(gt, trace)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("C", [2, 4, 8, 16])
@pytest.mark.parametrize("which", ["tiny", "fsm"])
def test_cluster_trace_and_results(C, which):
    _check(which, good_cluster=C)


@pytest.mark.parametrize("C", [2, 16])
def test_cluster_delay_chain(C):
    """Registers latching registers: each latch must read Q of the same cycle."""
    _check("chain", good_cluster=C)


@pytest.mark.parametrize("C", [4])
@pytest.mark.parametrize("window", [64, 128])
def test_cluster_windowed_resume(C, window):
    """Windows start the cluster trace at t_begin > 0 from the previous window's latch."""
    _check("fsm300", good_cluster=C, window=window)


@pytest.mark.parametrize("opts", [dict(), dict(good_cluster=2), dict(good_cluster=1), dict(window=64)])
def test_big_design_every_form(opts):
    """A design too large for one CTA's shared memory: automatic choice (a cluster), a
    forced cluster of 2 (levels wider than a chunk per CTA), one CTA over the global trace,
    and windows; trace and results equal the oracle's."""
    _check("big", **opts)


def test_cluster_batch_mixed_forms():
    """One campaign whose designs take different good-trace forms in the same window:
    small designs on single CTAs, the big one on a cluster."""
    designs = [synth.tiny_design(1), _big_design(), synth.gen_datapath_fsm(3, 3000, 300, 16, 16, [8], 0.8, 12, 64, "fsm3")]
    Ts = [100, 80, 150]
    stims = [synth.stimulus(d, T, 40 + i) for i, (d, T) in enumerate(zip(designs, Ts))]
    faults = [synth.sample_faults(d, 600, 50 + i) for i, d in enumerate(designs)]
    with Simulator(0) as sim:
        for d, s, f in zip(designs, stims, faults):
            sim.add(d, s, f)
        res, _ = sim.run(window=64)
        traces = [sim.good_trace(i) for i in range(len(designs))]
    for i, (d, s, f) in enumerate(zip(designs, stims, faults)):
        _, trace = oracle.good_run(d, s, with_trace=True)
        assert np.array_equal(traces[i], trace)
        exp = oracle.fault_sim(d, s, f, threads=8)
        for a, b in zip(split(res[i]), exp):
            assert np.array_equal(a, b)


def test_forced_cluster_size_errors():
    from paper_2508_16376_gb300.rtlfs import RtlfsError
    d = synth.tiny_design(1)
    with Simulator(0) as sim:
        sim.add(d, synth.stimulus(d, 20, 1), synth.sample_faults(d, 10, 1))
        for bad in (3, 32, -1):
            with pytest.raises(RtlfsError):
                sim.run(good_cluster=bad)
        sim.run(good_cluster=2)   # the context stays usable


@pytest.mark.parametrize("opts", [dict(), dict(window=64), dict(window=7), dict(use_graph=1)])
@pytest.mark.parametrize("which", ["tiny", "fsm", "chain", "big"])
def test_staged_good_trace(which, opts):
    """The staged one-CTA good trace (a producer warp copying each chunk's descriptors into
    a shared ring with bulk asynchronous copies) gives the oracle's trace and results: a
    design without nodes (no chunks at all), windows that resume mid-stimulus and end on a
    ragged cycle, graph replay, and a design whose net values only fit one CTA's shared
    memory without the ring (then on a cluster as before)."""
    _check(which, good_staging=1, **opts)


def test_staged_and_prefetched_forms_alternate():
    """Switching between the register-prefetched and the staged one-CTA trace on one
    context keeps the trace and the results."""
    d, stim, f, trace, exp = _case("fsm300")
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        for kw in (dict(good_staging=1), dict(), dict(good_staging=1, window=64), dict(window=64)):
            res, _ = sim.run(**kw)
            assert np.array_equal(sim.good_trace(0), trace), str(kw)
            for a, b in zip(split(res[0]), exp):
                assert np.array_equal(a, b), str(kw)
