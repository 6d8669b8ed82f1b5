"""The roofline's algorithmic counts, checked by hand on the 4-bit counter.

Counter: input 0 (8 b), Q (4 b), c = CONST (4 b), s = ADD(Q, c) (4 b), x = XOR(Q, c) (4 b);
5 nets, 3 nodes, all narrow. Ops per node (OPS + MASK): CONST 0 + 1, ADD 1 + 1, XOR 1 + 1
= 5 per good cycle; a faulty evaluation adds KEEP (1): (1 + 2 + 2 + 3) / 3 = 8/3 on average.
"""
import numpy as np

from paper_2508_16376_gb300 import roofline, synth


def test_counter_ops_and_bytes_by_hand():
    d = synth.counter4()
    T = 20
    stim = np.zeros((T, 1), np.uint64)
    f = synth.Faults(np.array([1, 2, 3], np.uint32), np.zeros(3, np.uint8), np.array([0, 1, 0], np.uint8))
    parts = [(d, stim, f)]
    assert roofline.node_ops(d) == (5, 8)
    stats = {"node_evals": 30, "fault_cycles": 45}
    ops = roofline.step_int_ops(parts, stats)
    assert ops == {"good": 5 * 20, "faulty": int(30 * 8 / 3), "output_check": 45,
                   "total": 100 + 80 + 45}
    # results: detected at cycle 0, undetected, detected at cycle 9 -> simulated 1, 20, 10 cycles
    res = [np.array([[1, 0, 1], [0, -1, 9], [0, -1, 0]])]
    # windows of 8 cycles: boundaries crossed = ceil(c/8) - 1 = 0, 2, 1
    assert roofline.crossings(parts, res, 8) == 3
    by = roofline.step_bytes(parts, res, {"window": 8})
    assert by == {"good_trace": 2 * 8 * 5 * 20, "stimulus": 8 * 1 * 20, "window_state": 30,
                  "faults": 3 * 25, "total": 1600 + 160 + 30 + 75}
    assert roofline.step_bytes(parts, res, {"window": 0})["window_state"] == 0
    assert roofline.windows({"window": 8}, 20) == 3 and roofline.windows({}, 20) == 1


def test_wide_nodes_take_the_wide_column():
    bld = synth._Builder([64], [])
    bld.add(synth.ADD, 64, 0, 0)        # 2 + 2
    bld.add(synth.CONCAT, 40, 0, 0)     # 4 + 2
    bld.add(synth.MUX2, 8, 0, 0, 0)     # 2 + 1
    d = bld.finish("w", [1])
    assert roofline.node_ops(d) == (4 + 6 + 3, (4 + 2) + (6 + 2) + (3 + 1))


def test_fractions_are_achieved_over_peak():
    d = synth.counter4()
    parts = [(d, np.zeros((20, 1), np.uint64), synth.Faults(np.array([1], np.uint32), np.zeros(1, np.uint8),
                                                            np.zeros(1, np.uint8)))]
    stats = {"node_evals": 10, "fault_cycles": 20}
    mean = {"good_ms": 0.1, "light_ms": 0.5, "heavy_ms": 0.2}
    ints = roofline.int_peak({}, 2000.0, 100)
    assert abs(ints["tops"] - 100 * roofline.INT32_LANES_PER_SM * 2e9 / 1e12) < 1e-12
    r = roofline.step_roofline(parts, None, stats, mean, {}, {"hbm_gbs": 1000.0}, 1, 1.0, ints)
    assert r["kernel"] == "light" and r["peak_source"] == "measured"
    assert abs(r["achieved"] - r["algorithmic_bytes_per_step"] / 0.5e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    a = roofline.step_alu(parts, stats, mean, 1, 1.0, ints)
    assert abs(a["frac"] - a["achieved"] / ints["tops"]) < 1e-12
    assert a["int_ops_per_step"] == roofline.step_int_ops(parts, stats)["total"]
    b = roofline.step_bound(r, a, 2.0)
    assert b["bound_s"] == max(r["algorithmic_bytes_per_step"] / 1e12, a["int_ops_per_step"] / (ints["tops"] * 1e12))
    assert abs(b["frac"] - b["bound_s"] / 2e-3) < 1e-12 and b["bound_by"] in ("hbm", "alu")
