"""GPU parity: every result of the CUDA path (through the C-ABI) equals the CPU oracle's,
bit-exact -- detected flag, first-detection cycle and first differing port -- and the good
trace equals the oracle's net by net. Sizes span many tiles, ragged tails, multiple
designs per launch, and every schedule knob (results must not depend on any of them)."""
import numpy as np
import pytest

import oracle
import ppsfp
import test_oracle_pins as pins
from paper_2508_16376_gb300 import synth
from paper_2508_16376_gb300 import rtlfs
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def gpu_run(design, stim, faults, plain=False, want_load=False, **opts):
    with Simulator(0) as sim:
        sim.add(design, stim, faults)
        if plain:
            res = sim.run_plain()
            loads = None
        else:
            res, loads = sim.run(want_load=want_load, **opts)
        st = sim.stats()
    det, cyc, port = split(res[0])
    return det, cyc, port, (loads[0] if loads else None), st


def assert_same(got, exp, what=""):
    det, cyc, port = got[:3]
    odet, ocyc, oport = exp[:3]
    bad = np.nonzero((det != odet) | (cyc != ocyc) | (port != oport))[0]
    assert bad.size == 0, (f"{what}: {bad.size} mismatches, first {bad[:8]}: "
                           f"gpu {det[bad[:4]]},{cyc[bad[:4]]},{port[bad[:4]]} "
                           f"oracle {odet[bad[:4]]},{ocyc[bad[:4]]},{oport[bad[:4]]}")


def small_fsm_design(seed, n=3000, regs=300):
    return synth.gen_datapath_fsm(seed, n, regs, 16, 16, [8], 0.8, 12, 64, f"fsm{seed}")


# ---- good trace ----------------------------------------------------------------------

@pytest.mark.parametrize("maker,T", [(lambda: synth.tiny_design(1), 100),
                                     (lambda: small_fsm_design(3), 333),
                                     (lambda: synth.counter4(), 37)])
def test_good_trace_matches_oracle(maker, T):
    d = maker()
    stim = synth.stimulus(d, T, 11, 0.1)
    g, trace = oracle.good_run(d, stim, with_trace=True)
    with Simulator(0) as sim:
        sim.add(d, stim, synth.Faults(np.zeros(0, np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.uint8)))
        gt = sim.good_trace(0)
        go = sim.good_outputs(0)
    assert np.array_equal(gt, trace)
    assert np.array_equal(go, g)


def test_good_trace_global_memory_path():
    """A design too large for shared-memory net values, kept on one CTA (good_cluster=1),
    runs the variant whose net values live in the global trace."""
    d = synth.gen_datapath_fsm(5, 30000, 600, 32, 32, [16], 0.5, 20, 64, "big")
    stim = synth.stimulus(d, 64, 5)
    g, trace = oracle.good_run(d, stim, with_trace=True)
    with Simulator(0) as sim:
        sim.add(d, stim, synth.sample_faults(d, 10, 1))
        sim.run(good_cluster=1)
        assert np.array_equal(sim.good_trace(0), trace)


# ---- fault simulation vs oracle ------------------------------------------------------

OPTION_SETS = [
    dict(),
    dict(heavy_frac=1.0, heavy_form=2),
    dict(heavy_frac=0.3, heavy_form=2, heavy_block=128),
    dict(heavy_frac=1.0, heavy_form=3),
    dict(heavy_frac=0.2, heavy_form=3, heavy_ctas=5),
    dict(scheduler=rtlfs.SCHED_PLAIN),
    dict(heavy_frac=0.05),
    dict(heavy_frac=1.0),
    dict(light_block=32, heavy_block=32),
    dict(light_block=256, heavy_block=512, heavy_frac=0.2),
    dict(heavy_ctas=3, heavy_frac=0.3),
]


@pytest.mark.parametrize("opts", OPTION_SETS)
def test_tiny_all_faults(opts):
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 100, 101)
    u = synth.fault_universe(d, include_inputs=True)
    exp = oracle.fault_sim(d, stim, u, threads=8)
    got = gpu_run(d, stim, u, **opts)
    assert_same(got, exp, f"tiny {opts}")


def test_tiny_plain_form():
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 100, 101)
    u = synth.fault_universe(d)
    exp = oracle.fault_sim(d, stim, u, threads=8)
    assert_same(gpu_run(d, stim, u, plain=True), exp, "plain")


@pytest.mark.parametrize("T", [20, 5])
def test_counter_golden_gpu(T):
    rows = pins._load_counter_golden()
    rows = rows[rows[:, 0] == T]
    f = synth.Faults(rows[:, 1].astype(np.uint32), rows[:, 2].astype(np.uint8), rows[:, 3].astype(np.uint8))
    stim = np.zeros((T, 1), np.uint64)
    for kw in (dict(), dict(heavy_frac=1.0)):
        det, cyc, port = gpu_run(synth.counter4(), stim, f, **kw)[:3]
        assert np.array_equal(det, rows[:, 4]) and np.array_equal(cyc, rows[:, 5])
        assert np.array_equal(port, rows[:, 6])


def test_delay_chain_gpu():
    d = synth.delay_chain(4, 12)
    stim = synth.stimulus(d, 64, 9)
    u = synth.fault_universe(d, include_inputs=True)
    assert_same(gpu_run(d, stim, u), oracle.fault_sim(d, stim, u), "delay")
    assert_same(gpu_run(d, stim, u, heavy_frac=1.0), oracle.fault_sim(d, stim, u), "delay heavy")


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bruteforce_gpu(seed):
    rng = np.random.default_rng(700 + seed)
    widths = [int(x) for x in rng.integers(1, 5, 3)]
    while sum(widths) > 11:
        widths.pop()
    d = synth.gen_comb_dag(100 + seed, n_nodes=40, input_widths=widths, n_outputs=3, node_wmax=8)
    stim = ppsfp.exhaustive_stimulus(d)
    u = synth.fault_universe(d, include_inputs=True)
    exp = ppsfp.brute_force(d, u)
    assert_same(gpu_run(d, stim, u), exp, "ppsfp")


@pytest.mark.parametrize("seed", [21, 22])
def test_fsm_design_all_faults_with_promotion(seed):
    """Datapath + FSM shape (heavy-tailed cones) at a size the oracle finishes quickly;
    the light kernel's capacities overflow on some faults, which must then finish
    bit-exact in the heavy kernel."""
    d = small_fsm_design(seed)
    stim = synth.stimulus(d, 400, seed, 0.1)
    u = synth.sample_faults(d, 4000, seed)
    exp = oracle.fault_sim(d, stim, u, threads=16)
    got = gpu_run(d, stim, u, want_load=True)
    assert_same(got, exp, "fsm")
    assert got[4]["promoted"] > 0
    for kw in (dict(heavy_frac=0.1), dict(scheduler=rtlfs.SCHED_PLAIN), dict(heavy_frac=1.0),
               dict(heavy_frac=1.0, heavy_form=2), dict(heavy_frac=1.0, heavy_form=1, window=64)):
        assert_same(gpu_run(d, stim, u, **kw), exp, f"fsm {kw}")


def test_batch_of_designs_one_launch():
    """Several designs of different sizes, cycle counts and fault counts (one empty) run in
    one rtlfs_run; each matches its own oracle run."""
    cases = []
    for i, (n, T, F) in enumerate([(800, 150, 900), (2500, 77, 1500), (200, 300, 0), (1200, 1, 500)]):
        d = small_fsm_design(40 + i, n, max(48, n // 10))
        stim = synth.stimulus(d, T, 40 + i, 0.1)
        f = synth.sample_faults(d, F, 40 + i) if F else synth.Faults(
            np.zeros(0, np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.uint8))
        cases.append((d, stim, f))
    with Simulator(0) as sim:
        for d, stim, f in cases:
            sim.add(d, stim, f)
        res, _ = sim.run(heavy_frac=0.05)
        res_p = sim.run_plain()
    for k, (d, stim, f) in enumerate(cases):
        exp = oracle.fault_sim(d, stim, f, threads=8)
        assert_same(split(res[k]), exp, f"batch {k}")
        assert_same(split(res_p[k]), exp, f"batch plain {k}")


def test_permuted_node_order():
    d = synth.tiny_design(5)
    stim = synth.stimulus(d, 60, 5)
    u = synth.fault_universe(d)
    rng = np.random.default_rng(1)
    perm = rng.permutation(d.n_node)
    base = d.n_in + d.n_reg
    newpos = np.empty(d.n_node, np.int64)
    newpos[perm] = np.arange(d.n_node)

    def ren(x):
        x = np.asarray(x, np.int64)
        return np.where(x >= base, base + newpos[np.maximum(x - base, 0)], x).astype(np.uint32)

    p = synth.Design("perm", d.input_widths, d.reg_widths, ren(d.reg_d), d.node_op[perm],
                     d.node_w[perm], ren(d.node_a[perm]), ren(d.node_b[perm]),
                     ren(d.node_c[perm]), d.node_imm[perm], ren(d.outputs))
    up = synth.Faults(ren(u.net), u.bit, u.val)
    assert_same(gpu_run(p, stim, up), oracle.fault_sim(d, stim, u, threads=8), "perm")


def test_duplicate_faults():
    d = synth.tiny_design(2)
    stim = synth.stimulus(d, 50, 2)
    u = synth.sample_faults(d, 300, 2)
    dup = synth.Faults.concat([u, u, u])
    det, cyc, port = gpu_run(d, stim, dup)[:3]
    for k in (1, 2):
        assert np.array_equal(det[:300], det[300 * k:300 * (k + 1)])
        assert np.array_equal(cyc[:300], cyc[300 * k:300 * (k + 1)])


def test_heavy_forms_alternate_on_one_context():
    """The exact and stamped heavy forms share their scratch: alternating them in one
    context (and windows with one pass) gives the same results and loads every time."""
    d = small_fsm_design(29)
    stim = synth.stimulus(d, 260, 29, 0.1)
    u = synth.sample_faults(d, 2500, 29)
    exp = oracle.fault_sim(d, stim, u, threads=16)
    with Simulator(0) as sim:
        sim.add(d, stim, u)
        ref = None
        for kw in (dict(heavy_form=1), dict(heavy_form=2), dict(heavy_form=1, window=64),
                   dict(heavy_form=2, window=64), dict(heavy_form=2), dict(heavy_form=1),
                   dict(heavy_form=3), dict(heavy_form=3, window=64), dict(heavy_form=1, window=64),
                   dict(heavy_form=3), dict(heavy_form=2)):
            res, loads = sim.run(want_load=True, heavy_frac=1.0, **kw)
            assert_same(split(res[0]), exp, str(kw))
            if ref is None:
                ref = loads[0]
            assert np.array_equal(loads[0], ref), str(kw)


def test_loads_are_schedule_independent():
    """The recorded propagation load of a fault is a property of the fault, not of the
    kernel that simulated it (the same nodes are evaluated in the same cycles)."""
    d = small_fsm_design(23)
    stim = synth.stimulus(d, 300, 23, 0.1)
    u = synth.sample_faults(d, 2000, 23)
    a = gpu_run(d, stim, u, want_load=True, heavy_frac=0.0)[3]
    b = gpu_run(d, stim, u, want_load=True, heavy_frac=1.0)[3]
    c = gpu_run(d, stim, u, want_load=True, heavy_frac=1.0, heavy_form=2)[3]
    e = gpu_run(d, stim, u, want_load=True, heavy_frac=1.0, heavy_form=3)[3]
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, e)
    assert a.sum() > 0


# ---- errors and budget -----------------------------------------------------------------

def _ctx():
    return rtlfs.rtlfs_create(0)


def test_error_codes():
    ctx = _ctx()
    try:
        good = synth.tiny_design(1)
        nodes, regs, iw, outs = rtlfs.design_arrays(good)
        bad = nodes.copy()
        bad[0]["width"] = 65
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_load_design(ctx, bad, regs, iw, outs)
        assert e.value.code == rtlfs.RTLFS_E_WIDTH
        bad = nodes.copy()
        bad[3]["a"] = good.n_net + 5
        bad[3]["op"] = synth.AND
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_load_design(ctx, bad, regs, iw, outs)
        assert e.value.code == rtlfs.RTLFS_E_ARG
        loop = synth._Builder([4], [])
        loop.add(synth.AND, 4, 0, 2)
        loop.add(synth.OR, 4, 1, 0)
        ld = loop.finish("loop", [1])
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_load_design(ctx, *rtlfs.design_arrays(ld))
        assert e.value.code == rtlfs.RTLFS_E_CYCLE
        did = rtlfs.rtlfs_load_design(ctx, nodes, regs, iw, outs)
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_run(ctx, [0])
        assert e.value.code == rtlfs.RTLFS_E_STATE
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_set_stimulus(ctx, did, np.zeros((0, good.n_in), np.uint64))
        assert e.value.code == rtlfs.RTLFS_E_ARG
        fa = rtlfs.fault_array(synth.sample_faults(good, 10, 1))
        fa[0]["bit"] = 63
        fa[0]["net"] = good.n_in   # a register of width <= 32
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_set_faults(ctx, did, fa)
        assert e.value.code == rtlfs.RTLFS_E_ARG
        with pytest.raises(rtlfs.RtlfsError) as e:
            rtlfs.rtlfs_set_faults(ctx, 7, fa)
        assert e.value.code == rtlfs.RTLFS_E_ARG
        # the context stays usable after the rejected calls
        rtlfs.rtlfs_set_stimulus(ctx, did, synth.stimulus(good, 30, 1))
        rtlfs.rtlfs_set_faults(ctx, did, rtlfs.fault_array(synth.sample_faults(good, 50, 1)))
        for bad_opts in (dict(good_staging=2), dict(heavy_form=4), dict(heavy_form=3, heavy_block=64)):
            with pytest.raises(rtlfs.RtlfsError) as e:
                rtlfs.rtlfs_run(ctx, [50], rtlfs.make_opts(**bad_opts))
            assert e.value.code == rtlfs.RTLFS_E_ARG
        res, _, _ = rtlfs.rtlfs_run(ctx, [50])
        assert len(res[0]) == 50
    finally:
        rtlfs.rtlfs_destroy(ctx)


def test_fault_budget_timeout_then_recovery():
    d = small_fsm_design(24)
    stim = synth.stimulus(d, 300, 24, 0.1)
    u = synth.sample_faults(d, 1500, 24)
    exp = oracle.fault_sim(d, stim, u, threads=8)
    with Simulator(0) as sim:
        sim.add(d, stim, u)
        res, loads, rc = rtlfs.rtlfs_run(sim.ctx, sim.n_faults, rtlfs.make_opts(fault_budget=50),
                                         want_load=True, check=False)
        assert rc == rtlfs.RTLFS_E_TIMEOUT
        det = res[0]["detected"]
        hit = det == 255
        assert hit.any()
        ok = ~hit
        assert np.array_equal(det[ok], exp[0][ok]) and np.array_equal(res[0]["cycle"][ok], exp[1][ok])
        res2, _ = sim.run()
        assert_same(split(res2[0]), exp, "after budget")


def test_cuda_graph_capture_and_replay():
    """use_graph: the first run captures the launch sequence, later runs replay it; a new
    fault list (new buffers) forces a new capture. Every result equals the oracle's."""
    d = small_fsm_design(25)
    stim = synth.stimulus(d, 300, 25, 0.1)
    u1 = synth.sample_faults(d, 2000, 25)
    u2 = synth.sample_faults(d, 2500, 26)
    e1 = oracle.fault_sim(d, stim, u1, threads=16)
    e2 = oracle.fault_sim(d, stim, u2, threads=16)
    with Simulator(0) as sim:
        sim.add(d, stim, u1)
        for _ in range(3):
            res, _ = sim.run(use_graph=1, heavy_frac=0.05)
            assert_same(split(res[0]), e1, "graph replay")
        sim.set_faults(0, u2)
        for _ in range(2):
            res, _ = sim.run(use_graph=1, heavy_frac=0.05)
            assert_same(split(res[0]), e2, "graph after new faults")
        res, _ = sim.run(use_graph=0)
        assert_same(split(res[0]), e2, "no graph")


# ---- windowed campaign ------------------------------------------------------------------

@pytest.mark.parametrize("window", [1, 7, 64, 300])
def test_windowed_matches_oracle(window):
    """Every live fault advances through the same window of cycles; light survivors carry
    their register diffs, heavy survivors go through the pool, promotions start in the
    window they happen in. Window sizes from 1 cycle to the whole stimulus, ragged ends."""
    d = small_fsm_design(27)
    stim = synth.stimulus(d, 257, 27, 0.1)
    u = synth.sample_faults(d, 3000, 27)
    exp = oracle.fault_sim(d, stim, u, threads=16)
    for kw in (dict(), dict(heavy_frac=0.1), dict(scheduler=rtlfs.SCHED_PLAIN, light_cap=1),
               dict(heavy_frac=1.0), dict(heavy_frac=1.0, heavy_form=2), dict(heavy_form=2, heavy_block=64),
               dict(heavy_frac=1.0, heavy_form=3), dict(heavy_frac=0.1, heavy_form=3)):
        got = gpu_run(d, stim, u, want_load=True, window=window, **kw)
        assert_same(got, exp, f"window {window} {kw}")
    ref = gpu_run(d, stim, u, want_load=True)
    assert np.array_equal(got[3], ref[3])      # same evaluations, windowed or not


def test_windowed_batch_and_graph():
    cases = []
    for i, (n, T, F) in enumerate([(900, 130, 800), (2200, 61, 1200), (300, 200, 0), (1500, 1, 400)]):
        d = small_fsm_design(60 + i, n, max(48, n // 10))
        stim = synth.stimulus(d, T, 60 + i, 0.1)
        f = synth.sample_faults(d, F, 60 + i) if F else synth.Faults(
            np.zeros(0, np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.uint8))
        cases.append((d, stim, f))
    with Simulator(0) as sim:
        for d, stim, f in cases:
            sim.add(d, stim, f)
        runs = [sim.run(window=32, heavy_frac=0.05)[0], sim.run(window=32, use_graph=1)[0],
                sim.run(window=32, use_graph=1)[0], sim.run(window=50, use_graph=1, light_cap=1)[0]]
    for k, (d, stim, f) in enumerate(cases):
        exp = oracle.fault_sim(d, stim, f, threads=8)
        for res in runs:
            assert_same(split(res[k]), exp, f"windowed batch {k}")


def test_windowed_counter_golden():
    rows = pins._load_counter_golden()
    rows = rows[rows[:, 0] == 20]
    f = synth.Faults(rows[:, 1].astype(np.uint32), rows[:, 2].astype(np.uint8), rows[:, 3].astype(np.uint8))
    stim = np.zeros((20, 1), np.uint64)
    for w in (1, 3, 8):
        det, cyc, port = gpu_run(synth.counter4(), stim, f, window=w, heavy_frac=0.5)[:3]
        assert np.array_equal(det, rows[:, 4]) and np.array_equal(cyc, rows[:, 5])
        assert np.array_equal(port, rows[:, 6])
