"""Checkpoint and resume of a windowed campaign: a run stopped at a window boundary, its
state saved to bytes, loaded into a fresh context and resumed, reaches the uninterrupted
run's results, loads, counters and no-drop mismatch counts, and both equal the oracle. The
stopped run's own results are final for every fault it no longer simulates; the rest report
RTLFS_PENDING. Malformed or mismatched checkpoints are refused."""
import functools

import numpy as np
import pytest

import oracle
from paper_2508_16376_gb300 import rtlfs, synth
from paper_2508_16376_gb300.rtlfs import RTLFS_PENDING, RtlfsError, Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _with_cycles(f):
    if f.cycle is None:
        f = synth.Faults(f.net, f.bit, f.val, np.zeros(len(f), np.uint32))
    return f


@functools.lru_cache(maxsize=None)
def _designs():
    """Two designs of different lengths in one context: a multi-cycle FSM datapath with
    stuck-at, transient and port faults (T = 333, ragged last window), and the tiny design
    (T = 100, finished before the later stop cycles)."""
    d0 = synth.gen_datapath_fsm(3, 3000, 300, 16, 16, [8], 0.8, 12, 64, "fsm3")
    s0 = synth.stimulus(d0, 333, 11, 0.1)
    f0 = _with_cycles(synth.Faults.concat([synth.sample_faults(d0, 1500, 9),
                                           synth.transient_faults(d0, 600, 333, 5),
                                           synth.port_faults(d0)]))
    d1 = synth.tiny_design(1)
    s1 = synth.stimulus(d1, 100, 101)
    f1 = _with_cycles(synth.Faults.concat([synth.fault_universe(d1),
                                           synth.transient_faults(d1, 300, 100, 6)]))
    return [(d0, s0, f0), (d1, s1, f1)]


@functools.lru_cache(maxsize=None)
def _oracle(no_drop):
    return [oracle.fault_sim_ex(d, s, f, threads=16, no_drop=no_drop) for d, s, f in _designs()]


def _sim(n=2):
    sim = Simulator(0)
    for d, s, f in _designs()[:n]:
        sim.add(d, s, f)
    return sim


def _full(n, **opts):
    with _sim(n) as sim:
        res, loads = sim.run(want_load=True, **opts)
        cnt = [sim.mismatch_counts(i) for i in range(n)] if opts.get("no_drop") else None
        return res, loads, sim.stats(), cnt


def _check_stopped(res, final, stop, no_drop):
    """Non-pending results are final; pending faults are the ones not finished by `stop`
    (with no_drop, detected faults stay alive too)."""
    for r, fr in zip(res, final):
        pend = r["detected"] == RTLFS_PENDING
        done = ~pend
        assert np.array_equal(r[done], fr[done])
        assert np.all(r["cycle"][pend] == -1) and np.all(r["port"][pend] == -1)
        if not no_drop:   # a fault detected before the stop was final there
            early = (fr["detected"] == 1) & (fr["cycle"] < stop)
            assert not np.any(pend & early)


OPTS = [dict(window=64, heavy_frac=0.3), dict(window=64, heavy_frac=0.0, light_cap=1),
        dict(window=64, heavy_frac=1.0, heavy_form=2), dict(window=128, heavy_frac=0.3, no_drop=1),
        dict(window=64, heavy_frac=0.3, no_drop=1, heavy_form=1), dict(window=64, heavy_frac=1.0, heavy_form=3)]


@pytest.mark.parametrize("opts", OPTS)
@pytest.mark.parametrize("stops", [(64,), (128,), (320,), (64, 192)])
def test_stop_save_load_resume(opts, stops):
    W = opts["window"]
    if any(s % W for s in stops):
        pytest.skip("stop cycles must be multiples of the window")
    no_drop = bool(opts.get("no_drop"))
    full_res, full_loads, full_st, full_cnt = _full(2, **opts)
    # the uninterrupted run agrees with the oracle
    for r, e in zip(full_res, _oracle(no_drop)):
        for a, b in zip(split(r), e[:3]):
            assert np.array_equal(a, b)
    blob = None
    for i, stop in enumerate(stops):
        with _sim() as sim:
            if blob is not None:
                sim.restore(blob)
            res, _ = sim.run(stop_cycle=stop, resume=1 if blob is not None else 0, **opts)
            _check_stopped(res, full_res, stop, no_drop)
            blob = sim.checkpoint()
            assert len(blob) == rtlfs.rtlfs_checkpoint_size(sim.ctx)
    with _sim() as sim:
        sim.restore(blob)
        res, loads = sim.run(want_load=True, resume=1, **opts)
        st = sim.stats()
        cnt = [sim.mismatch_counts(i) for i in range(2)] if no_drop else None
    for a, b in zip(res, full_res):
        assert np.array_equal(a, b)
    for a, b in zip(loads, full_loads):
        assert np.array_equal(a, b)
    for k in ("node_evals", "fault_cycles"):
        assert st[k] == full_st[k], k
    # each fault's evaluations are counted once, by the kernel that kept them; which faults
    # start in the heavy kernel is decided among equal predicted loads by arrival order, so
    # only the sums are fixed unless every fault starts on one side
    assert st["light_evals"] + st["heavy_evals"] == full_st["light_evals"] + full_st["heavy_evals"]
    assert (st["light_fault_cycles"] + st["heavy_fault_cycles"]
            == full_st["light_fault_cycles"] + full_st["heavy_fault_cycles"])
    if opts["heavy_frac"] in (0.0, 1.0):
        for k in ("light_evals", "light_fault_cycles", "heavy_evals", "heavy_fault_cycles"):
            assert st[k] == full_st[k], k
    if no_drop:
        for a, b, e in zip(cnt, full_cnt, _oracle(True)):
            assert np.array_equal(a, b)
            assert np.array_equal(a, e[3])


def test_resume_in_same_context():
    opts = dict(window=64, heavy_frac=0.3)
    full_res, full_loads, _, _ = _full(2, **opts)
    with _sim() as sim:
        sim.run(stop_cycle=128, **opts)
        res, loads = sim.run(want_load=True, resume=1, **opts)
        # the checkpoint is used up by a run that reaches the end
        with pytest.raises(RtlfsError):
            sim.run(resume=1, **opts)
    for a, b in zip(res, full_res):
        assert np.array_equal(a, b)
    for a, b in zip(loads, full_loads):
        assert np.array_equal(a, b)


def test_stopped_counts_refused_until_end():
    with _sim() as sim:
        sim.run(stop_cycle=64, window=64, no_drop=1)
        with pytest.raises(RtlfsError):
            sim.mismatch_counts(0)


def test_checkpoint_errors():
    opts = dict(window=64, heavy_frac=0.3)
    with _sim() as sim:
        with pytest.raises(RtlfsError):          # nothing to resume from
            sim.run(resume=1, **opts)
        with pytest.raises(RtlfsError):          # no checkpoint held
            sim.checkpoint()
        for bad in (dict(stop_cycle=100), dict(stop_cycle=384), dict(stop_cycle=-64),
                    dict(stop_cycle=64, use_graph=1), dict(stop_cycle=64, window=0)):
            with pytest.raises(RtlfsError):
                sim.run(**{**opts, **bad})
        sim.run(stop_cycle=128, **opts)
        blob = sim.checkpoint()
        with pytest.raises(RtlfsError):          # other window
            sim.run(resume=1, **{**opts, "window": 32})
        with pytest.raises(RtlfsError):          # other no-drop mode
            sim.run(resume=1, no_drop=1, **opts)
        with pytest.raises(RtlfsError):          # stop not after the checkpoint
            sim.run(resume=1, stop_cycle=128, **opts)
        # a changed fault list drops the checkpoint
        d, s, f = _designs()[0]
        sim.set_faults(0, f)
        with pytest.raises(RtlfsError):
            sim.run(resume=1, **opts)
    with _sim() as sim:
        with pytest.raises(RtlfsError):
            sim.restore(b"\0" * 16)
        with pytest.raises(RtlfsError):
            sim.restore(blob[:-8])
        with pytest.raises(RtlfsError):
            sim.restore(b"XXXXXXXX" + blob[8:])
    with _sim(1) as sim:                         # other designs
        with pytest.raises(RtlfsError):
            sim.restore(blob)
    with Simulator(0) as sim:                    # other fault list
        for i, (d, s, f) in enumerate(_designs()):
            sim.add(d, s, f.take(np.arange(len(f) - 1)) if i == 1 else f)
        with pytest.raises(RtlfsError):
            sim.restore(blob)
    with _sim() as sim:                          # a good blob still loads after the refusals
        sim.restore(blob)
        res, _ = sim.run(resume=1, **opts)
    full_res, _, _, _ = _full(2, **opts)
    for a, b in zip(res, full_res):
        assert np.array_equal(a, b)


def _layout(blob):
    """Offsets of the checkpoint fields (the saved layout: a 56-byte header, then the per-design
    and per-fault arrays in a fixed order)."""
    h = np.frombuffer(blob[:56], np.uint8)
    u32 = h[8:40].view(np.uint32)
    nd, F, n_live, n_carry = int(u32[0]), int(u32[1]), int(u32[5]), int(u32[6])
    pool_top = int(h[40:48].view(np.uint64)[0])
    off, o = {}, 56
    for name, size in (("T", 4 * nd), ("n_net", 4 * nd), ("det", F), ("cycle", 4 * F), ("port", 4 * F),
                       ("load", 8 * F), ("mism", 4 * F), ("st_nreg", F), ("st_r", 32 * F), ("st_v", 64 * F),
                       ("live", 4 * n_live), ("carry", 16 * n_carry), ("pool_r", 4 * pool_top)):
        off[name] = o
        o += size
    return off, F, n_live, n_carry, pool_top


def test_checkpoint_contents_checked():
    """A loaded checkpoint is checked against the kernels' bounds: a live light fault with
    more register diffs than its light capacity holds, a carried heavy fault naming a
    register outside its design, and a resume under another light capacity are refused."""
    opts = dict(window=64, heavy_frac=0.3, light_cap=1)
    with _sim() as sim:
        sim.run(stop_cycle=64, **opts)
        blob = sim.checkpoint()
        with pytest.raises(RtlfsError):          # other light capacity
            sim.run(resume=1, **{**opts, "light_cap": 2})
    off, F, n_live, n_carry, pool_top = _layout(blob)
    assert n_live > 0
    live0 = int(np.frombuffer(blob, np.uint32, 1, off["live"])[0])
    bad = bytearray(blob)
    bad[off["st_nreg"] + live0] = 5               # light capacity 1 holds 4
    with _sim() as sim:
        with pytest.raises(RtlfsError):
            sim.restore(bytes(bad))
    carry0 = np.frombuffer(blob, np.uint32, 4, off["carry"]) if n_carry else np.zeros(4, np.uint32)
    if int(carry0[1]) > 0:                        # nreg of the first carry
        bad = bytearray(blob)
        pos = off["pool_r"] + 4 * int(np.frombuffer(blob, np.uint64, 1, off["carry"] + 8)[0])
        bad[pos:pos + 4] = np.uint32(0xFFFFFF).tobytes()
        with _sim() as sim:
            with pytest.raises(RtlfsError):
                sim.restore(bytes(bad))
    with _sim() as sim:                           # the untouched blob resumes
        sim.restore(blob)
        res, _ = sim.run(resume=1, **opts)
    full_res, _, _, _ = _full(2, **opts)
    for a, b in zip(res, full_res):
        assert np.array_equal(a, b)
