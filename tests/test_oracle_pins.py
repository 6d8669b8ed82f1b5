"""Pins of the CPU oracle to facts that do not come from the oracle itself.

* a hand-derived 4-bit counter (tests/golden/counter4.txt);
* a register delay chain whose detection cycles have a closed form in the stimulus;
* exhaustive brute force on small combinational designs by parallel-pattern
  single-fault propagation over truth-table bitsets (tests/ppsfp.py), whose word-level
  ops are rebuilt from single-bit logic;
* invariants of the stuck-at problem: no path to an output => never detected; stuck
  value equal to the good value in every cycle => never detected; stimulus prefix;
  duplicated descriptors; node order does not matter (the oracle sorts topologically).
"""
import os

import numpy as np
import pytest

import oracle
import ppsfp
from paper_2508_16376_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load_counter_golden():
    rows = []
    with open(os.path.join(GOLDEN, "counter4.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return np.array(rows, np.int64)


@pytest.mark.parametrize("T", [20, 5])
def test_counter4_golden(T):
    d = synth.counter4()
    rows = _load_counter_golden()
    rows = rows[rows[:, 0] == T]
    assert len(rows) == 32
    stim = np.zeros((T, 1), np.uint64)
    g = oracle.good_outputs(d, stim)
    assert list(g[:, 0]) == [t % 16 for t in range(T)]
    f = synth.Faults(rows[:, 1].astype(np.uint32), rows[:, 2].astype(np.uint8),
                     rows[:, 3].astype(np.uint8))
    det, cyc, port = oracle.fault_sim(d, stim, f)
    assert np.array_equal(det, rows[:, 4])
    assert np.array_equal(cyc, rows[:, 5])
    assert np.array_equal(port, rows[:, 6])


def test_counter4_universe_matches_golden_sites():
    u = synth.fault_universe(synth.counter4())
    assert len(u) == 32
    assert set(np.unique(u.net)) == {1, 2, 3, 4}


def test_register_truncates_wider_d():
    """3-bit register Q latching the 4-bit s = ADD(Q, CONST 1): the latch keeps the low
    3 bits, so the good output Q is t mod 8 (hand-derived), and a stuck-at on s's bit 3
    never reaches Q (undetected either way). Q[2] SA0 shows at the first t with bit 2
    set, t = 4; s[0] SA0 makes Q stick at 0, seen at t = 1."""
    bld = synth._Builder([8], [3])
    c = bld.add(synth.CONST, 4, imm=1)
    s = bld.add(synth.ADD, 4, bld.reg_net(0), c)
    bld.reg_d[0] = s
    d = bld.finish("wrap3", [bld.reg_net(0)])
    T = 20
    stim = np.zeros((T, 1), np.uint64)
    assert list(oracle.good_outputs(d, stim)[:, 0]) == [t % 8 for t in range(T)]
    f = synth.Faults(np.array([s, s, 1, s], np.uint32), np.array([3, 3, 2, 0], np.uint8),
                     np.array([1, 0, 0, 0], np.uint8))
    det, cyc, port = oracle.fault_sim(d, stim, f)
    assert list(det) == [0, 0, 1, 1]
    assert list(cyc) == [-1, -1, 4, 1]


def _delay_expected(stim_col, k, site, bit, val, T):
    """Closed form for delay_chain(k): output at t is reg_k's Q = input[t-k] (0 before).
    A fault on input 0 or on reg_j's Q (site = j, 0 for the input) forces that bit at the
    point it is produced; downstream registers copy it, so the faulty output at t is
    0 for t < k-j, force(0) for k-j <= t < k and force(input[t-k]) for t >= k."""
    j = site

    def force(x):
        return (x & ~(1 << bit)) | (val << bit)

    for t in range(T):
        good = 0 if t < k else int(stim_col[t - k])
        if t < k - j:
            bad = 0                      # registers downstream of the site still hold reset 0
        elif t < k:
            bad = force(0)               # reg_j's forced reset value has reached the output
        else:
            bad = force(int(stim_col[t - k]))
        if bad != good:
            return 1, t, 0
    return 0, -1, -1


@pytest.mark.parametrize("k,width,seed", [(1, 8, 3), (3, 8, 4), (5, 16, 5)])
def test_delay_chain_closed_form(k, width, seed):
    d = synth.delay_chain(k, width)
    T = 48
    stim = synth.stimulus(d, T, seed)
    col = stim[:, 0] & np.uint64((1 << width) - 1)
    u = synth.fault_universe(d, include_inputs=True)
    det, cyc, port = oracle.fault_sim(d, stim, u)
    for f in range(len(u)):
        site = int(u.net[f])               # 0 = input, 1..k = reg_1..reg_k
        exp = _delay_expected(col, k, site, int(u.bit[f]), int(u.val[f]), T)
        assert (int(det[f]), int(cyc[f]), int(port[f])) == exp, (f, site, exp)


@pytest.mark.parametrize("seed", list(range(8)))
def test_brute_force_combinational(seed):
    rng = np.random.default_rng(500 + seed)
    widths = [int(x) for x in rng.integers(1, 5, int(rng.integers(2, 4)))]
    while sum(widths) > 11:
        widths.pop()
    d = synth.gen_comb_dag(seed, n_nodes=int(rng.integers(12, 30)), input_widths=widths,
                           n_outputs=int(rng.integers(1, 4)), node_wmax=8)
    stim = ppsfp.exhaustive_stimulus(d)
    u = synth.fault_universe(d, include_inputs=True)
    det, cyc, port = oracle.fault_sim(d, stim, u)
    bdet, bcyc, bport = ppsfp.brute_force(d, u)
    assert np.array_equal(det, bdet)
    assert np.array_equal(cyc, bcyc)
    assert np.array_equal(port, bport)
    # the good outputs agree too
    good_bits, _ = ppsfp.evaluate(d)
    g = oracle.good_outputs(d, stim)
    for o, net in enumerate(d.outputs):
        vals = np.zeros(stim.shape[0], np.uint64)
        for i, bsv in enumerate(good_bits[int(net)]):
            for p in range(stim.shape[0]):
                if (bsv >> p) & 1:
                    vals[p] |= np.uint64(1 << i)
        assert np.array_equal(vals, g[:, o])


def test_brute_force_covers_every_op():
    """The brute-force designs above draw ops at random; this one has each op at least
    once, every operand a distinct input so that a transposed operand changes results."""
    bld = synth._Builder([3, 3, 2], [])
    a, b, s = 0, 1, 2
    outs = []
    for op in (synth.AND, synth.OR, synth.XOR, synth.ADD, synth.SUB, synth.EQ, synth.LT):
        outs.append(bld.add(op, 4 if op not in (synth.EQ, synth.LT) else 1, a, b))
    outs.append(bld.add(synth.NOT, 4, a))
    outs.append(bld.add(synth.MUX2, 3, s, a, b))
    outs.append(bld.add(synth.SHL, 5, a, imm=2))
    outs.append(bld.add(synth.SHR, 3, a, imm=1))
    outs.append(bld.add(synth.SLICE, 2, b, imm=1))
    outs.append(bld.add(synth.CONCAT, 5, a, s))
    cst = bld.add(synth.CONST, 3, imm=5)
    outs.append(bld.add(synth.SUB, 3, cst, b))
    outs.append(bld.add(synth.SHL, 4, b, imm=70))
    d = bld.finish("allops", outs)
    stim = ppsfp.exhaustive_stimulus(d)
    u = synth.fault_universe(d, include_inputs=True)
    det, cyc, port = oracle.fault_sim(d, stim, u)
    bdet, bcyc, bport = ppsfp.brute_force(d, u)
    assert np.array_equal(det, bdet) and np.array_equal(cyc, bcyc) and np.array_equal(port, bport)
    assert det.mean() > 0.5


def _reaches_output(d):
    """Static reachability to any output through node operands and register D->Q edges."""
    users = [[] for _ in range(d.n_net)]
    base = d.n_in + d.n_reg
    nops = {synth.CONST: 0, synth.NOT: 1, synth.SHL: 1, synth.SHR: 1, synth.SLICE: 1, synth.MUX2: 3}
    for i in range(d.n_node):
        k = nops.get(int(d.node_op[i]), 2)
        for x in [int(d.node_a[i]), int(d.node_b[i]), int(d.node_c[i])][:k]:
            users[x].append(base + i)
    for r in range(d.n_reg):
        users[int(d.reg_d[r])].append(d.n_in + r)
    seen = np.zeros(d.n_net, bool)
    stack = [int(o) for o in d.outputs]
    # walk backwards: a net reaches an output if some user reaches one
    rev = [[] for _ in range(d.n_net)]
    for x in range(d.n_net):
        for u in users[x]:
            rev[u].append(x)
    while stack:
        n = stack.pop()
        if seen[n]:
            continue
        seen[n] = True
        stack.extend(rev[n])
    return seen


def test_invariants_tiny():
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 100, 101)
    u = synth.fault_universe(d, include_inputs=True)
    g, trace = oracle.good_run(d, stim, with_trace=True)
    det, cyc, port = oracle.fault_sim(d, stim, u, threads=4, gout=g)
    reach = _reaches_output(d)
    unreach = ~reach[u.net]
    assert unreach.any()
    assert not det[unreach].any()                      # invariant 1
    bitvals = (trace[:, u.net] >> u.bit.astype(np.uint64)) & np.uint64(1)
    always_eq = (bitvals == u.val[None, :].astype(np.uint64)).all(axis=0)
    assert always_eq.any()
    assert not det[always_eq].any()                    # invariant 2
    # detected faults report a port that observes a differing value; ports are in range
    assert (port[det == 1] >= 0).all() and (port[det == 1] < d.n_out).all()
    assert ((cyc >= 0) == (det == 1)).all()


def test_prefix_and_duplicates():
    d = synth.tiny_design(3)
    stim = synth.stimulus(d, 80, 7)
    u = synth.sample_faults(d, 1500, 9)
    det, cyc, port = oracle.fault_sim(d, stim, u, threads=4)
    for Tp in (1, 17, 40):
        d2, c2, p2 = oracle.fault_sim(d, stim[:Tp], u, threads=4)
        early = (det == 1) & (cyc < Tp)
        assert np.array_equal(d2.astype(bool), early)
        assert np.array_equal(c2[early], cyc[early]) and np.array_equal(p2[early], port[early])
    dup = synth.Faults.concat([u.take(np.arange(50)), u.take(np.arange(50))])
    dd, dc, dp = oracle.fault_sim(d, stim, dup)
    assert np.array_equal(dd[:50], dd[50:]) and np.array_equal(dc[:50], dc[50:])
    assert np.array_equal(dd[:50], det[:50]) and np.array_equal(dc[:50], cyc[:50])


def test_node_order_irrelevant():
    """Permuting the node list (with operands renamed) changes no result."""
    d = synth.tiny_design(5)
    stim = synth.stimulus(d, 60, 5)
    u = synth.fault_universe(d)
    det, cyc, port = oracle.fault_sim(d, stim, u, threads=4)
    rng = np.random.default_rng(0)
    perm = rng.permutation(d.n_node)           # new position -> old node
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
    d2, c2, p2 = oracle.fault_sim(p, stim, up, threads=4)
    assert np.array_equal(det, d2) and np.array_equal(cyc, c2) and np.array_equal(port, p2)


def test_combinational_cycle_rejected():
    bld = synth._Builder([4], [])
    bld.add(synth.AND, 4, 0, 2)     # node 0 reads node 1 (net 2)
    bld.add(synth.OR, 4, 1, 0)      # node 1 reads node 0 (net 1)
    d = bld.finish("loop", [1])
    assert oracle.topo_order(d) is None
    with pytest.raises(ValueError):
        oracle.good_outputs(d, np.zeros((3, 1), np.uint64))
