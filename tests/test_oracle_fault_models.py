"""Pins of the oracle's other fault models (transient SEU/SET flips, output-port faults
through a virtual node) and of its no-drop mode (mismatch-cycle counts), each against
something other than the oracle: hand-derived counter results (tests/golden), closed forms
on register delay chains, exhaustive truth-table brute force on combinational designs, and
invariants tying the no-drop mode to the dropping one."""
import os

import numpy as np
import pytest

import oracle
import ppsfp
from paper_2508_16376_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "counter4_extended.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x) for x in line.split()])
    return np.array(rows, np.int64)


def test_counter4_extended_golden():
    r = _rows()
    d = synth.counter4()
    for T in sorted(set(r[:, 0].tolist())):
        rr = r[r[:, 0] == T]
        stim = np.zeros((T, 1), np.uint64)
        f = synth.Faults(rr[:, 2].astype(np.uint32), rr[:, 3].astype(np.uint8), rr[:, 1].astype(np.uint8),
                         rr[:, 4].astype(np.uint32))
        det, cyc, port, cnt = oracle.fault_sim_ex(d, stim, f, no_drop=True)
        assert np.array_equal(det, rr[:, 5]) and np.array_equal(cyc, rr[:, 6])
        assert np.array_equal(port, rr[:, 7]) and np.array_equal(cnt, rr[:, 8])
        # dropping: the same first detection, a detected fault counts its one cycle
        det2, cyc2, port2, cnt2 = oracle.fault_sim_ex(d, stim, f, no_drop=False)
        assert np.array_equal(det2, det) and np.array_equal(cyc2, cyc) and np.array_equal(port2, port)
        assert np.array_equal(cnt2, det.astype(np.uint32))


@pytest.mark.parametrize("k,w,T", [(1, 8, 30), (4, 5, 30), (9, 13, 40)])
def test_delay_chain_transient_closed_form(k, w, T):
    """A flip of reg_r (0-based) in cycle c reaches the output (reg_{k-1}'s Q) in cycle
    c + (k-1-r); a flip of the input in cycle c is latched at its end and arrives in
    cycle c + k. The pulse is seen once."""
    d = synth.delay_chain(k, w)
    rng = np.random.default_rng(k * 100 + w)
    stim = rng.integers(0, 1 << w, (T, 1)).astype(np.uint64)
    nets, bits, kinds, cycles, expect = [], [], [], [], []
    for r in range(k):
        for c in (0, 3, T - 1 - (k - 1 - r), T - (k - 1 - r), T + 7):
            nets.append(1 + r); bits.append(int(rng.integers(0, w))); kinds.append(2); cycles.append(max(c, 0))
            arrive = max(c, 0) + (k - 1 - r)
            expect.append(arrive if arrive < T else -1)
    for c in (0, 5, T - 1 - k, T - k, T):
        nets.append(0); bits.append(int(rng.integers(0, w))); kinds.append(3); cycles.append(c)
        expect.append(c + k if c + k < T else -1)
    f = synth.Faults(np.array(nets, np.uint32), np.array(bits, np.uint8), np.array(kinds, np.uint8),
                     np.array(cycles, np.uint32))
    det, cyc, port, cnt = oracle.fault_sim_ex(d, stim, f, no_drop=True)
    expect = np.array(expect)
    assert np.array_equal(cyc, expect)
    assert np.array_equal(det, (expect >= 0).astype(np.uint8))
    assert np.array_equal(cnt, (expect >= 0).astype(np.uint32))


def _comb_design(seed):
    rng = np.random.default_rng(seed)
    widths = [int(x) for x in rng.integers(1, 5, 3)]
    while sum(widths) > 11:
        widths[int(np.argmax(widths))] -= 1
    return synth.gen_comb_dag(seed, 24, widths, 4)


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_fault_models(seed):
    """Stuck-at (with no-drop counts), SET flips at chosen vectors and port faults on a
    combinational design against parallel-pattern brute force over every input vector."""
    d = _comb_design(seed)
    stim = ppsfp.exhaustive_stimulus(d)
    P = stim.shape[0]
    rng = np.random.default_rng(seed)
    sa = synth.fault_universe(d, include_inputs=True)
    sa = sa.take(rng.choice(len(sa), min(len(sa), 120), replace=False))
    ports = synth.port_faults(d)
    widths = d.net_widths()
    n_set = 80
    nets = rng.integers(0, d.n_net, n_set)
    set_f = synth.Faults(nets.astype(np.uint32), (rng.random(n_set) * widths[nets]).astype(np.uint8),
                         np.full(n_set, 3, np.uint8), rng.integers(0, P + 2, n_set).astype(np.uint32))
    pn = rng.integers(0, d.n_out, 20)
    pw = widths[np.asarray(d.outputs, np.int64)[pn]]
    pset = synth.Faults((pn + d.n_net).astype(np.uint32), (rng.random(20) * pw).astype(np.uint8),
                        np.full(20, 3, np.uint8), rng.integers(0, P, 20).astype(np.uint32))
    for f in (sa, ports, set_f, pset):
        if f.cycle is None:
            f = synth.Faults(f.net, f.bit, f.val, np.zeros(len(f), np.uint32))
        got = oracle.fault_sim_ex(d, stim, f, no_drop=True)
        exp = ppsfp.brute_force_ex(d, f)
        for a, b in zip(got, exp):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", [3, 4])
def test_nodrop_invariants_sequential(seed):
    """On a sequential design: the no-drop first detection equals the dropping result, a
    fault is counted iff detected, the count fits in the cycles after the detection; a
    port fault is detected exactly where the fault function changes the port's good value
    (closed form from the good outputs)."""
    d = synth.gen_datapath_fsm(seed, 600, 80, 8, 8, [8], 0.8, 8, 32, f"s{seed}")
    T = 120
    stim = synth.stimulus(d, T, seed, 0.1)
    f = synth.sample_faults(d, 300, seed)
    f = synth.Faults.concat([f, synth.transient_faults(d, 200, T, seed), synth.port_faults(d)])
    det, cyc, port, cnt = oracle.fault_sim_ex(d, stim, f, no_drop=True)
    det2, cyc2, port2, _ = oracle.fault_sim_ex(d, stim, f, no_drop=False)
    assert np.array_equal(det, det2) and np.array_equal(cyc, cyc2) and np.array_equal(port, port2)
    assert np.array_equal(cnt > 0, det == 1)
    assert np.all(cnt[det == 1] <= T - cyc[det == 1])
    g = oracle.good_outputs(d, stim)
    is_port = f.net >= d.n_net
    for i in np.nonzero(is_port)[0]:
        o = int(f.net[i]) - d.n_net
        b = (g[:, o] >> np.uint64(f.bit[i])) & np.uint64(1)
        kind = int(f.val[i])
        if kind <= 1:
            hits = np.nonzero(b != kind)[0]
        else:
            c = int(f.cycle[i])
            hits = np.array([c]) if c < T else np.zeros(0, np.int64)
        assert cnt[i] == len(hits)
        assert cyc[i] == (hits[0] if len(hits) else -1)
