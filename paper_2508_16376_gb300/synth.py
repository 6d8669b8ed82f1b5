"""Seeded synthetic workloads: word-level RTL op graphs, stimuli and stuck-at fault lists.

This module only *builds inputs*; it evaluates nothing. Both the CUDA path (through the
C-ABI) and the CPU oracle receive the same arrays from it, so it holds none of the
simulator's arithmetic (no op evaluation, no masking of values, no detection logic).

The paper's benchmark designs, stimuli and fault lists (Table II: RISCV Mini, Conv Acc,
Sodor, PicoRV32, GEMM, JPEG, Conv2D) are not available, so the workloads here are
synthetic stand-ins with the same shape: a levelized word-level graph of RTL nodes
(Sec. II-B, Fig. 2), registers latched at the end of every cycle (global
synchronization, Sec. II-B), stuck-at-0/1 faults on wires and registers (Sec. IV-A,
Sec. V-A), and a control FSM whose bits steer datapath multiplexers, which gives the
few-heavy / many-light load split the paper measures (Sec. III, Fig. 4).

Net id space of a design: [0, I) primary inputs, [I, I+R) register Q outputs,
[I+R, I+R+N) node outputs (node i drives net I+R+i).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Op codes of the word-level graph; the same numbering is declared in include/rtlfs.h.
AND, OR, XOR, NOT, ADD, SUB, MUX2, EQ, LT, SHL, SHR, SLICE, CONCAT, CONST = range(14)
OP_NAMES = ["AND", "OR", "XOR", "NOT", "ADD", "SUB", "MUX2", "EQ", "LT", "SHL", "SHR",
            "SLICE", "CONCAT", "CONST"]
DATAPATH_OPS = [AND, OR, XOR, NOT, ADD, SUB, MUX2, EQ, LT, SHL, SHR, SLICE, CONCAT]


@dataclasses.dataclass
class Design:
    """A word-level op graph in the layout the C-ABI takes (structure of arrays)."""
    name: str
    input_widths: np.ndarray   # uint8 [I]
    reg_widths: np.ndarray     # uint8 [R]
    reg_d: np.ndarray          # uint32 [R]  net id latched into the register
    node_op: np.ndarray        # uint8 [N]
    node_w: np.ndarray         # uint8 [N]
    node_a: np.ndarray         # uint32 [N]
    node_b: np.ndarray         # uint32 [N]
    node_c: np.ndarray         # uint32 [N]
    node_imm: np.ndarray       # uint64 [N]
    outputs: np.ndarray        # uint32 [O]  output port o observes net outputs[o]
    control_nets: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros(0, np.uint32))   # FSM/control nets (reporting only)

    @property
    def n_in(self) -> int:
        return int(self.input_widths.shape[0])

    @property
    def n_reg(self) -> int:
        return int(self.reg_widths.shape[0])

    @property
    def n_node(self) -> int:
        return int(self.node_op.shape[0])

    @property
    def n_out(self) -> int:
        return int(self.outputs.shape[0])

    @property
    def n_net(self) -> int:
        return self.n_in + self.n_reg + self.n_node

    def net_widths(self) -> np.ndarray:
        return np.concatenate([self.input_widths, self.reg_widths, self.node_w]).astype(np.uint8)

    def save(self, path: str) -> None:
        np.savez(path, **{f.name: getattr(self, f.name) for f in dataclasses.fields(self)})

    @staticmethod
    def load(path: str) -> "Design":
        z = np.load(path, allow_pickle=False)
        kw = {f.name: z[f.name] for f in dataclasses.fields(Design)}
        kw["name"] = str(kw["name"])
        return Design(**kw)


@dataclasses.dataclass
class Faults:
    """Fault descriptors: bit `bit` of net `net` (ids n_net + o: output port o). `val` is
    the kind: 0 / 1 stuck-at 0 / 1, 2 an SEU (register) and 3 an SET (input, node or port)
    flipping the bit in cycle `cycle` (None: every fault is a stuck-at)."""
    net: np.ndarray   # uint32 [F]
    bit: np.ndarray   # uint8 [F]
    val: np.ndarray   # uint8 [F]
    cycle: Optional[np.ndarray] = None   # uint32 [F]

    def __len__(self) -> int:
        return int(self.net.shape[0])

    def take(self, idx) -> "Faults":
        return Faults(self.net[idx], self.bit[idx], self.val[idx],
                      None if self.cycle is None else self.cycle[idx])

    @staticmethod
    def concat(parts: Sequence["Faults"]) -> "Faults":
        cyc = None
        if any(p.cycle is not None for p in parts):
            cyc = np.concatenate([p.cycle if p.cycle is not None else np.zeros(len(p), np.uint32)
                                  for p in parts]).astype(np.uint32)
        return Faults(np.concatenate([p.net for p in parts]).astype(np.uint32),
                      np.concatenate([p.bit for p in parts]).astype(np.uint8),
                      np.concatenate([p.val for p in parts]).astype(np.uint8), cyc)


class _Builder:
    """Incremental graph builder; nodes are appended in a topological order."""

    def __init__(self, input_widths: Sequence[int], reg_widths: Sequence[int]):
        self.I = len(input_widths)
        self.R = len(reg_widths)
        self.in_w = list(int(w) for w in input_widths)
        self.reg_w = list(int(w) for w in reg_widths)
        self.reg_d = [0] * self.R
        self.op: List[int] = []
        self.w: List[int] = []
        self.a: List[int] = []
        self.b: List[int] = []
        self.c: List[int] = []
        self.imm: List[int] = []
        self.widths: List[int] = self.in_w + self.reg_w   # width of every net so far

    def reg_net(self, r: int) -> int:
        return self.I + r

    def add(self, op: int, w: int, a: int = 0, b: int = 0, c: int = 0, imm: int = 0) -> int:
        self.op.append(op)
        self.w.append(int(w))
        self.a.append(int(a))
        self.b.append(int(b))
        self.c.append(int(c))
        self.imm.append(int(imm))
        net = self.I + self.R + len(self.op) - 1
        self.widths.append(int(w))
        return net

    def finish(self, name: str, outputs: Sequence[int], control: Sequence[int] = ()) -> Design:
        return Design(
            name=name,
            input_widths=np.asarray(self.in_w, np.uint8),
            reg_widths=np.asarray(self.reg_w, np.uint8),
            reg_d=np.asarray(self.reg_d, np.uint32),
            node_op=np.asarray(self.op, np.uint8),
            node_w=np.asarray(self.w, np.uint8),
            node_a=np.asarray(self.a, np.uint32),
            node_b=np.asarray(self.b, np.uint32),
            node_c=np.asarray(self.c, np.uint32),
            node_imm=np.asarray(self.imm, np.uint64),
            outputs=np.asarray(list(outputs), np.uint32),
            control_nets=np.asarray(list(control), np.uint32),
        )


def _add_fsm(bld: _Builder, rng: np.random.Generator, state_regs: Sequence[int]) -> List[int]:
    """One-hot FSM over 1-bit registers `state_regs`, built only from the op set.

    State j advances to j+1 when its guard (EQ or LT on a 2-3 bit input slice against a
    constant) holds, otherwise jumps to a random state when a second guard holds, else
    stays. All registers reset to 0, so state 0's next-state term also ORs in
    NOT(OR-reduce of every state bit): the FSM enters state 0 at cycle 1.
    Returns the state Q nets (the control bits the datapath reads).
    """
    S = len(state_regs)
    q = [bld.reg_net(r) for r in state_regs]

    def guard() -> int:
        k = int(rng.integers(bld.I))
        wk = bld.in_w[k]
        sw = int(min(wk, rng.integers(2, 4)))
        lo = int(rng.integers(0, wk - sw + 1))
        sl = bld.add(SLICE, sw, k, imm=lo)
        cst = bld.add(CONST, sw, imm=int(rng.integers(0, 1 << sw)))
        if rng.random() < 0.5:
            return bld.add(EQ, 1, sl, cst)
        return bld.add(LT, 1, sl, cst)

    incoming: List[List[int]] = [[] for _ in range(S)]
    stay: List[int] = []
    for j in range(S):
        g1 = guard()
        g2 = guard()
        n1 = bld.add(NOT, 1, g1)
        adv = bld.add(AND, 1, q[j], g1)
        jmp = bld.add(AND, 1, q[j], bld.add(AND, 1, n1, g2))
        st = bld.add(AND, 1, q[j], bld.add(AND, 1, n1, bld.add(NOT, 1, g2)))
        incoming[(j + 1) % S].append(adv)
        incoming[int(rng.integers(S))].append(jmp)
        stay.append(st)
    # OR-reduce of the state bits (balanced tree), then the reset-entry term.
    level = list(q)
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            nxt.append(bld.add(OR, 1, level[i], level[i + 1]))
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    none_hot = bld.add(NOT, 1, level[0])
    for j in range(S):
        terms = [stay[j]] + incoming[j] + ([none_hot] if j == 0 else [])
        acc = terms[0]
        for t in terms[1:]:
            acc = bld.add(OR, 1, acc, t)
        bld.reg_d[state_regs[j]] = acc
    return q


def _random_node(bld: _Builder, rng: np.random.Generator, pick, wmax: int,
                 sel_pool: Optional[Sequence[int]], sel_p: float) -> int:
    """Append one datapath node with a uniformly drawn op; operands come from `pick()`."""
    op = DATAPATH_OPS[int(rng.integers(len(DATAPATH_OPS)))]
    W = bld.widths
    if op in (EQ, LT):
        return bld.add(op, 1, pick(), pick())
    if op == SLICE:
        a = pick()
        wa = W[a]
        w = int(rng.integers(1, wa + 1))
        lo = int(rng.integers(0, wa - w + 1))
        return bld.add(SLICE, w, a, imm=lo)
    if op == CONCAT:
        for _ in range(8):
            a, b = pick(), pick()
            if W[a] + W[b] <= wmax:
                return bld.add(CONCAT, W[a] + W[b], a, b)
        op = XOR   # no operand pair narrow enough: fall back to a two-input op
    w = int(rng.integers(1, wmax + 1))
    if op == NOT:
        return bld.add(NOT, w, pick())
    if op in (SHL, SHR):
        return bld.add(op, w, pick(), imm=int(rng.integers(0, w + 1)))
    if op == MUX2:
        if sel_pool is not None and len(sel_pool) and rng.random() < sel_p:
            s = int(sel_pool[int(rng.integers(len(sel_pool)))])
        else:
            s = pick()
        return bld.add(MUX2, w, s, pick(), pick())
    return bld.add(op, w, pick(), pick())


def gen_random_dag(seed: int, n_nodes: int = 200, n_regs: int = 16, n_inputs: int = 8,
                   n_outputs: int = 8, in_width: int = 8, node_wmax: int = 32,
                   reg_wmin: int = 8, reg_wmax: int = 32, name: str = "tiny") -> Design:
    """Random DAG: operands drawn uniformly from every earlier net (inputs, register Qs,
    nodes). Register D inputs are random node outputs; outputs are random nodes or regs."""
    rng = np.random.default_rng(seed)
    reg_w = [int(x) for x in rng.integers(reg_wmin, reg_wmax + 1, n_regs)]
    bld = _Builder([in_width] * n_inputs, reg_w)

    def pick() -> int:
        return int(rng.integers(len(bld.widths)))

    for _ in range(n_nodes):
        _random_node(bld, rng, pick, node_wmax, None, 0.0)
    first_node = bld.I + bld.R
    for r in range(n_regs):
        bld.reg_d[r] = int(rng.integers(first_node, first_node + n_nodes))
    outs = [int(x) for x in rng.integers(bld.I, bld.I + bld.R + n_nodes, n_outputs)]
    return bld.finish(name, outs)


def gen_comb_dag(seed: int, n_nodes: int, input_widths: Sequence[int], n_outputs: int,
                 node_wmax: int = 8) -> Design:
    """Purely combinational random DAG (no registers), for exhaustive brute force."""
    rng = np.random.default_rng(seed)
    bld = _Builder(list(input_widths), [])

    def pick() -> int:
        return int(rng.integers(len(bld.widths)))

    for _ in range(n_nodes):
        _random_node(bld, rng, pick, node_wmax, None, 0.0)
    outs = [int(x) for x in rng.integers(bld.I, bld.I + n_nodes, n_outputs)]
    return bld.finish(f"comb{seed}", outs)


def gen_datapath_fsm(seed: int, n_nodes: int, n_regs: int, n_inputs: int, n_outputs: int,
                     fsm_states: Sequence[int], fsm_stage_frac: float, n_stages: int,
                     wmax: int = 64, name: str = "medium") -> Design:
    """Pipelined datapath steered by one-hot FSMs (the medium/large/batch shape).

    The datapath is `n_stages` stages; a node in stage s reads mostly stage s-1 and s-2
    nets (preferring ones nobody reads yet), register Qs and inputs. A fraction
    `fsm_stage_frac` of the stages belongs to one of the FSMs: their MUX2 selects are that
    FSM's state bits. Registers latch nodes of the last stages; outputs observe the last
    stage and some registers. Node count includes the FSM logic.
    """
    rng = np.random.default_rng(seed)
    fsm_regs_total = int(sum(fsm_states))
    assert fsm_regs_total < n_regs
    in_w = [int(x) for x in rng.integers(8, wmax + 1, n_inputs)]
    reg_w = [1] * fsm_regs_total + [int(x) for x in rng.integers(1, wmax + 1, n_regs - fsm_regs_total)]
    bld = _Builder(in_w, reg_w)

    fsm_q: List[List[int]] = []
    r0 = 0
    for S in fsm_states:
        fsm_q.append(_add_fsm(bld, rng, list(range(r0, r0 + S))))
        r0 += S
    control = [n for q in fsm_q for n in q]
    dp_regs = list(range(fsm_regs_total, n_regs))
    n_dp = n_nodes - len(bld.op)
    assert n_dp > n_stages

    stage_fsm = []
    for _ in range(n_stages):
        stage_fsm.append(int(rng.integers(len(fsm_q))) if (fsm_q and rng.random() < fsm_stage_frac) else -1)
    bounds = np.linspace(0, n_dp, n_stages + 1).astype(int)
    stage_nets: List[List[int]] = []
    unread = set()
    reg_nets = [bld.reg_net(r) for r in dp_regs]

    for s in range(n_stages):
        prev1 = stage_nets[s - 1] if s >= 1 else []
        prev2 = stage_nets[s - 2] if s >= 2 else []
        pool_unread = [n for n in prev1 if n in unread]

        def pick() -> int:
            u = rng.random()
            if prev1 and u < 0.55:
                if pool_unread and rng.random() < 0.6:
                    i = int(rng.integers(len(pool_unread)))
                    n = pool_unread[i]
                    pool_unread[i] = pool_unread[-1]
                    pool_unread.pop()
                else:
                    n = prev1[int(rng.integers(len(prev1)))]
            elif prev2 and u < 0.70:
                n = prev2[int(rng.integers(len(prev2)))]
            elif u < 0.88 or not prev1:
                if rng.random() < 0.7:
                    n = reg_nets[int(rng.integers(len(reg_nets)))]
                else:
                    n = int(rng.integers(bld.I))
            else:
                n = int(rng.integers(bld.I + bld.R, len(bld.widths)))   # any earlier node
            unread.discard(n)
            return n

        sel = fsm_q[stage_fsm[s]] if stage_fsm[s] >= 0 else None
        nets = []
        for _ in range(bounds[s + 1] - bounds[s]):
            n = _random_node(bld, rng, pick, wmax, sel, 0.9)
            nets.append(n)
            unread.add(n)
        stage_nets.append(nets)

    # Registers latch nodes of the last quarter of the stages, unread ones first.
    tail = [n for st in stage_nets[-max(1, n_stages // 4):] for n in st]
    tail_unread = [n for n in tail if n in unread]
    rng.shuffle(tail_unread)
    for i, r in enumerate(dp_regs):
        if i < len(tail_unread) and rng.random() < 0.8:
            d = tail_unread[i]
        else:
            d = tail[int(rng.integers(len(tail)))]
        bld.reg_d[r] = d
        unread.discard(d)
    # Outputs: 3/4 from the last stage (unread first), 1/4 register Qs.
    last = stage_nets[-1]
    last_unread = [n for n in last if n in unread]
    rng.shuffle(last_unread)
    outs = []
    n_reg_out = n_outputs // 4
    for i in range(n_outputs - n_reg_out):
        outs.append(last_unread[i] if i < len(last_unread) else last[int(rng.integers(len(last)))])
    for _ in range(n_reg_out):
        outs.append(reg_nets[int(rng.integers(len(reg_nets)))])
    return bld.finish(name, outs, control)


# ---- the five workload shapes -------------------------------------------------------

def tiny_design(seed: int = 1) -> Design:
    """200 nodes, widths 1-32, 16 regs of 8-32 b, 8 inputs of 8 b, 8 outputs."""
    return gen_random_dag(seed, 200, 16, 8, 8, 8, 32, 8, 32, "tiny")


def medium_design(seed: int = 2) -> Design:
    """20k nodes, 2k regs of 1-64 b, 64 inputs, 64 outputs, one 32-state one-hot FSM
    steering the MUX2 selects of most datapath stages."""
    return gen_datapath_fsm(seed, 20000, 2000, 64, 64, [32], 0.8, 40, 64, "medium")


def large_design(seed: int = 4) -> Design:
    """200k nodes, 20k regs of 1-64 b, 256 inputs, 256 outputs, 8 FSMs of 16-64 states
    steering 30% of the datapath stages."""
    rng = np.random.default_rng(seed + 7919)
    states = [int(x) for x in rng.integers(16, 65, 8)]
    return gen_datapath_fsm(seed, 200000, 20000, 256, 256, states, 0.3, 64, 64, "large")


def batch_designs(seed0: int = 1000, count: int = 64) -> List[Tuple[Design, int, int]]:
    """`count` designs, nodes log-uniform in [1k, 50k] with the medium shape; each with
    its own cycle count T uniform in [1k, 20k] and fault count F uniform in [5k, 50k].
    Returns (design, T, F) triples; design i uses seed seed0 + i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(math.exp(rng.uniform(math.log(1000), math.log(50000)))))
        T = int(rng.integers(1000, 20001))
        F = int(rng.integers(5000, 50001))
        regs = max(48, n // 10)
        stages = int(max(8, min(40, n // 250)))
        d = gen_datapath_fsm(seed0 + i, n, regs, 64, 64, [32], 0.8, stages, 64, f"batch{i}")
        out.append((d, T, F))
    return out


# ---- stimulus and faults ------------------------------------------------------------

def stimulus(design: Design, T: int, seed: int, hold_p: float = 0.0) -> np.ndarray:
    """[T, I] uint64 input vectors: uniform random bits (the consumer masks each to its
    input width); with probability hold_p a cycle repeats the previous vector whole
    (cycle 0 is always fresh)."""
    rng = np.random.default_rng(seed)
    raw = rng.bit_generator.random_raw(T * design.n_in).astype(np.uint64).reshape(T, design.n_in)
    if hold_p > 0 and T > 1:
        hold = rng.random(T) < hold_p
        hold[0] = False
        src = np.arange(T)
        src[hold] = 0
        src = np.maximum.accumulate(np.where(hold, 0, src))
        raw = raw[src]
    return np.ascontiguousarray(raw)


def fault_universe(design: Design, include_inputs: bool = False) -> Faults:
    """SA0 and SA1 on every bit of every node output and register Q output (and of every
    primary input when include_inputs); ordered by net, bit, stuck value."""
    widths = design.net_widths().astype(np.int64)
    first = 0 if include_inputs else design.n_in
    nets = np.arange(first, design.n_net, dtype=np.int64)
    w = widths[first:]
    net_rep = np.repeat(nets, w)
    starts = np.repeat(np.cumsum(w) - w, w)
    bits = np.arange(int(w.sum()), dtype=np.int64) - starts
    net2 = np.repeat(net_rep, 2)
    bit2 = np.repeat(bits, 2)
    val2 = np.tile(np.array([0, 1], np.int64), net_rep.shape[0])
    return Faults(net2.astype(np.uint32), bit2.astype(np.uint8), val2.astype(np.uint8))


def port_faults(design: Design) -> Faults:
    """SA0 and SA1 on every bit of every output port (net ids n_net + o: a virtual node
    between the port's net and the port); ordered by port, bit, stuck value."""
    widths = design.net_widths().astype(np.int64)
    w = widths[np.asarray(design.outputs, np.int64)]
    ports = np.arange(len(w), dtype=np.int64) + design.n_net
    net_rep = np.repeat(ports, w)
    starts = np.repeat(np.cumsum(w) - w, w)
    bits = np.arange(int(w.sum()), dtype=np.int64) - starts
    return Faults(np.repeat(net_rep, 2).astype(np.uint32), np.repeat(bits, 2).astype(np.uint8),
                  np.tile(np.array([0, 1], np.int64), net_rep.shape[0]).astype(np.uint8))


def transient_faults(design: Design, F: int, T: int, seed: int, port_share: float = 0.05) -> Faults:
    """F transient faults: SEUs on register bits (kind 2) and SETs on input, node and
    output-port bits (kind 3), each at a cycle uniform in [0, T]; cycle T never acts."""
    rng = np.random.default_rng(seed)
    widths = design.net_widths().astype(np.int64)
    n_port = int(round(F * port_share)) if design.n_out else 0
    nets = rng.integers(0, design.n_net, F - n_port)
    ports = rng.integers(0, max(design.n_out, 1), n_port) if n_port else np.zeros(0, np.int64)
    out_w = widths[np.asarray(design.outputs, np.int64)] if design.n_out else np.zeros(0, np.int64)
    net = np.concatenate([nets, ports + design.n_net]).astype(np.int64)
    w = np.concatenate([widths[nets], out_w[ports] if n_port else np.zeros(0, np.int64)])
    bit = (rng.random(F) * w).astype(np.int64)
    is_reg = (net >= design.n_in) & (net < design.n_in + design.n_reg)
    kind = np.where(is_reg, 2, 3)
    cycle = rng.integers(0, T + 1, F)
    return Faults(net.astype(np.uint32), bit.astype(np.uint8), kind.astype(np.uint8),
                  cycle.astype(np.uint32))


def sample_faults(design: Design, F: int, seed: int) -> Faults:
    """F faults drawn uniformly without replacement from the universe, kept in universe order."""
    u = fault_universe(design)
    if F >= len(u):
        return u
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(u), size=F, replace=False))
    return u.take(idx)


# ---- named workloads -----------------------------------------------------------------

def batch_workload(seed0: int = 1000, count: int = 64) -> List[Tuple[Design, np.ndarray, Faults]]:
    """The batched campaign: the `count` designs of batch_designs(seed0, count), design i
    with its own uniform random stimulus of T_i cycles (seed 1_000_000 + seed0 + i) and
    F_i stuck-at faults sampled from its universe (seed 2_000_000 + seed0 + i).
    Returns (design, stimulus, faults) triples."""
    out = []
    for i, (d, T, F) in enumerate(batch_designs(seed0, count)):
        out.append((d, stimulus(d, T, 1_000_000 + seed0 + i),
                    sample_faults(d, F, 2_000_000 + seed0 + i)))
    return out


def workload(name: str):
    """(design, stimulus, faults) for a named single-design workload shape: tiny (200
    nodes, full fault list), medium (20k nodes, 100k faults), large (200k nodes, 1M
    faults). The 64-design batch is batch_workload()."""
    if name == "tiny":
        d = tiny_design(1)
        return d, stimulus(d, 100, 101), fault_universe(d)
    if name == "medium":
        d = medium_design(2)
        return d, stimulus(d, 10000, 102, 0.1), sample_faults(d, 100000, 202)
    if name == "large":
        d = large_design(4)
        return d, stimulus(d, 20000, 104), sample_faults(d, 1000000, 204)
    raise ValueError(name)


# ---- hand-checkable fixtures ---------------------------------------------------------

def counter4() -> Design:
    """4-bit counter: Q (4-bit reg) <- s = ADD(Q, c), c = CONST 1 (4 b); one output = Q;
    a dangling x = XOR(Q, c) reaches no output; one unused 8-bit input.
    Net ids: input 0, Q 1, c 2, s 3, x 4."""
    bld = _Builder([8], [4])
    c = bld.add(CONST, 4, imm=1)
    s = bld.add(ADD, 4, bld.reg_net(0), c)
    bld.add(XOR, 4, bld.reg_net(0), c)
    bld.reg_d[0] = s
    return bld.finish("counter4", [bld.reg_net(0)])


def delay_chain(k: int, width: int) -> Design:
    """k registers in a chain: reg_1 latches input 0, reg_{i+1} latches reg_i's Q; the
    single output observes reg_k's Q. No nodes."""
    bld = _Builder([width], [width] * k)
    bld.reg_d[0] = 0
    for i in range(1, k):
        bld.reg_d[i] = bld.reg_net(i - 1)
    return bld.finish(f"delay{k}", [bld.reg_net(k - 1)])
