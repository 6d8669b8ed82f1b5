"""GPU parity for the other fault models and the no-drop mode: transient flips (SEU on
registers, SET on inputs, nodes and output ports), stuck-at faults on output ports
(virtual node), and no-drop runs with per-fault mismatch-cycle counts. Every form of the
path -- light lanes, heavy CTAs from cycle 0, windows, one pass, graph replay, cluster good
trace, plain form -- against the oracle, bit-exact, plus the hand-derived counter file."""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_2508_16376_gb300 import rtlfs, synth
from paper_2508_16376_gb300.rtlfs import RtlfsError, Simulator, split

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "counter4_extended.txt")

FORMS = [dict(), dict(window=32), dict(heavy_frac=1.0), dict(window=64, heavy_frac=0.3),
         dict(window=64, heavy_frac=1.0), dict(use_graph=1), dict(light_cap=1), dict(good_cluster=4),
         dict(window=64, heavy_frac=1.0, heavy_form=2), dict(heavy_frac=1.0, heavy_form=2),
         dict(window=64, heavy_frac=1.0, heavy_form=3), dict(heavy_frac=1.0, heavy_form=3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _run(d, stim, f, no_drop=False, plain=False, **opts):
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        if plain:
            res = sim.run_plain()
            cnt = None
        else:
            res, _ = sim.run(no_drop=1 if no_drop else 0, **opts)
            cnt = sim.mismatch_counts(0) if no_drop else None
    return split(res[0]), cnt


@functools.lru_cache(maxsize=None)
def _case(which):
    if which == "fsm":
        d = synth.gen_datapath_fsm(3, 3000, 300, 16, 16, [8], 0.8, 12, 64, "fsm3")
        T = 333
        stim = synth.stimulus(d, T, 11, 0.1)
        f = synth.Faults.concat([synth.transient_faults(d, 1500, T, 5), synth.port_faults(d),
                                 synth.sample_faults(d, 600, 9)])
    else:
        d = synth.tiny_design(1)
        T = 100
        stim = synth.stimulus(d, T, 101)
        f = synth.Faults.concat([synth.transient_faults(d, 800, T, 6), synth.port_faults(d),
                                 synth.fault_universe(d)])
    if f.cycle is None:
        f = synth.Faults(f.net, f.bit, f.val, np.zeros(len(f), np.uint32))
    drop = oracle.fault_sim_ex(d, stim, f, threads=16, no_drop=False)
    nodrop = oracle.fault_sim_ex(d, stim, f, threads=16, no_drop=True)
    return d, stim, f, drop, nodrop


@pytest.mark.parametrize("opts", FORMS)
@pytest.mark.parametrize("which", ["tiny", "fsm"])
def test_fault_models_drop(which, opts):
    d, stim, f, exp, _ = _case(which)
    got, _ = _run(d, stim, f, **opts)
    for a, b in zip(got, exp[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("opts", FORMS)
@pytest.mark.parametrize("which", ["tiny", "fsm"])
def test_fault_models_nodrop_counts(which, opts):
    d, stim, f, _, exp = _case(which)
    got, cnt = _run(d, stim, f, no_drop=True, **opts)
    for a, b in zip(got, exp[:3]):
        assert np.array_equal(a, b)
    assert np.array_equal(cnt, exp[3])


@pytest.mark.parametrize("which", ["tiny", "fsm"])
def test_fault_models_plain_form(which):
    d, stim, f, exp, _ = _case(which)
    got, _ = _run(d, stim, f, plain=True)
    for a, b in zip(got, exp[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("opts", [dict(), dict(window=0), dict(heavy_frac=1.0)])
def test_counter4_extended_golden_gpu(opts):
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x) for x in line.split()])
    r = np.array(rows, np.int64)
    d = synth.counter4()
    T = int(r[0, 0])
    f = synth.Faults(r[:, 2].astype(np.uint32), r[:, 3].astype(np.uint8), r[:, 1].astype(np.uint8),
                     r[:, 4].astype(np.uint32))
    (det, cyc, port), cnt = _run(d, np.zeros((T, 1), np.uint64), f, no_drop=True, **opts)
    assert np.array_equal(det, r[:, 5]) and np.array_equal(cyc, r[:, 6])
    assert np.array_equal(port, r[:, 7]) and np.array_equal(cnt, r[:, 8])


def test_transient_loads_schedule_independent():
    d, stim, f, _, _ = _case("fsm")
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        a = sim.run(want_load=True, heavy_frac=0.0)[1][0]
        b = sim.run(want_load=True, heavy_frac=1.0)[1][0]
    assert np.array_equal(a, b)


def test_mismatch_counts_state_and_errors():
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 30, 1)
    with Simulator(0) as sim:
        sim.add(d, stim, synth.sample_faults(d, 50, 1))
        sim.run()
        with pytest.raises(RtlfsError):          # the last run dropped faults
            sim.mismatch_counts(0)
        sim.run(no_drop=1)
        assert sim.mismatch_counts(0).shape == (50,)
        sim.set_faults(0, synth.sample_faults(d, 40, 2))
        with pytest.raises(RtlfsError):          # the list changed since
            sim.mismatch_counts(0)
        n_reg0 = d.n_in                          # first register net
        bad = [
            synth.Faults(np.array([n_reg0 - 1], np.uint32), np.zeros(1, np.uint8), np.array([2], np.uint8), np.zeros(1, np.uint32)),  # SEU on an input
            synth.Faults(np.array([n_reg0], np.uint32), np.zeros(1, np.uint8), np.array([3], np.uint8), np.zeros(1, np.uint32)),      # SET on a register
            synth.Faults(np.array([d.n_net + d.n_out], np.uint32), np.zeros(1, np.uint8), np.array([0], np.uint8), None),           # no such port
            synth.Faults(np.array([d.n_net], np.uint32), np.array([63], np.uint8), np.array([1], np.uint8), None),                   # bit beyond width
            synth.Faults(np.array([n_reg0], np.uint32), np.zeros(1, np.uint8), np.array([4], np.uint8), np.zeros(1, np.uint32)),      # unknown kind
        ]
        for f in bad:
            with pytest.raises(RtlfsError):
                sim.set_faults(0, f)
        sim.set_faults(0, synth.sample_faults(d, 10, 3))   # the context stays usable
        sim.run()
