"""The oracle pins are strong enough to catch plausible mistakes.

Each case compiles a copy of oracle/oracle_sim.c with one planted mistake (a dropped
term, a transposed operand, a wrong index or an off-by-one in the latch timing) into a
temporary directory, routes the oracle through it, and checks that at least one pin --
the hand-derived counter, the delay-chain closed form or the PPSFP brute force --
rejects it. Everything runs on the CPU.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import ppsfp
import test_oracle_fault_models as fm
import test_oracle_pins as pins
from paper_2508_16376_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle_sim.c")

MUTANTS = {
    "sub_operands_swapped": ("r[O_SUB]    = a - b;", "r[O_SUB]    = b - a;"),
    "lt_not_strict": ("r[O_LT]     = (a < b) ? 1 : 0;", "r[O_LT]     = (a <= b) ? 1 : 0;"),
    "mux_arms_swapped": ("r[O_MUX2]   = (a != 0) ? b : c;", "r[O_MUX2]   = (a != 0) ? c : b;"),
    "concat_halves_swapped": ("r[O_CONCAT] = (s->wb >= 64 ? 0 : (a << s->wb)) | b;",
                              "r[O_CONCAT] = (s->wb >= 64 ? 0 : (b << s->wb)) | a;"),
    "no_result_mask": ("return r[s->op] & s->mask;", "return r[s->op];"),
    "shr_as_shl": ("r[O_SHR]    = k >= 64 ? 0 : (a >> k);", "r[O_SHR]    = k >= 64 ? 0 : (a << k);"),
    "concat_width_of_a": ("s->wb = s->op == O_CONCAT ? net_width(d, d->b[i]) : 0;",
                          "s->wb = s->op == O_CONCAT ? net_width(d, d->a[i]) : 0;"),
    "no_force_on_reg_read": ("            net[I + r] = Q[r];\n            FORCE(I + r);",
                             "            net[I + r] = Q[r];"),
    "no_force_on_node": ("            net[st->out] = eval_step(st, net);\n            FORCE(st->out);",
                         "            net[st->out] = eval_step(st, net);"),
    "latch_without_mask": ("Q[r] = net[d->reg_d[r]] & mask_of(d->reg_w[r]);",
                           "Q[r] = net[d->reg_d[r]];"),
    "stuck_value_inverted": ("if (fault_val) m1 = (uint64_t)1 << fault_bit;",
                             "if (!fault_val) m1 = (uint64_t)1 << fault_bit;"),
    "highest_port_wins": ("for (int32_t o = 0; o < O; o++) {\n                uint64_t seen",
                          "for (int32_t o = O - 1; o >= 0; o--) {\n                uint64_t seen"),
    "flip_in_every_cycle": ("fx = (int64_t)t == fault_cycle ? mx : 0;", "fx = mx;"),
    "nodrop_counts_once": ("++*mism;", "*mism = 1;"),
    "port_fault_ignored": ("if ((int64_t)o == fault_port) seen = FAULTY(seen);", ""),
}


def _pins_pass() -> bool:
    try:
        for T in (20, 5):
            pins.test_counter4_golden(T)
        for args in [(1, 8, 3), (3, 8, 4)]:
            pins.test_delay_chain_closed_form(*args)
        for seed in range(4):
            pins.test_brute_force_combinational(seed)
        pins.test_brute_force_covers_every_op()
        pins.test_register_truncates_wider_d()
        _multi_port_pin()
        fm.test_counter4_extended_golden()
        fm.test_delay_chain_transient_closed_form(4, 5, 30)
        fm.test_brute_force_fault_models(0)
    except AssertionError:
        return False
    return True


def _multi_port_pin():
    """Two ports observe the same input bit, port 1 first in net order: a detection must
    name port 0 (ties go to the lowest port index)."""
    bld = synth._Builder([2], [])
    n1 = bld.add(synth.SLICE, 1, 0, imm=0)
    n2 = bld.add(synth.NOT, 1, n1)
    d = bld.finish("ports", [n2, n1])
    stim = ppsfp.exhaustive_stimulus(d)
    u = synth.fault_universe(d, include_inputs=True)
    det, cyc, port = oracle.fault_sim(d, stim, u)
    bdet, bcyc, bport = ppsfp.brute_force(d, u)
    assert np.array_equal(port, bport) and np.array_equal(cyc, bcyc)


def test_unmutated_oracle_passes():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", lib, str(path)])
    with oracle.use_library(lib):
        assert not _pins_pass(), f"mutant {name} survived every pin"
