"""Exhaustive brute force for combinational designs: parallel-pattern single-fault
propagation (PPSFP) over truth-table bitsets. Test pin for the oracle.

Every input vector of a design with n <= ~14 total input bits is applied at once: each
net bit is a 2^n-bit Python integer whose bit p is that net bit's value under input
vector p (p counts the vectors in order, so vector p is stimulus cycle p). The word-level
ops are rebuilt from single-bit logic -- ripple-carry addition, borrow-chain compare,
bit rewiring for shifts/slices/concatenation -- so this shares nothing with the oracle's
uint64 evaluator. One fault at a time is injected by overwriting one net bit with the
all-zeros or all-ones bitset (the stuck-at fault model, Sec. II-B) and the whole design
is re-evaluated; the first detecting vector is the lowest set bit of the OR of
(good XOR faulty) over all output bits (detection by comparing good and faulty output
values, Sec. II-B).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

import numpy as np

AND, OR, XOR, NOT, ADD, SUB, MUX2, EQ, LT, SHL, SHR, SLICE, CONCAT, CONST = range(14)


class Bitsets:
    def __init__(self, n_bits: int):
        self.P = 1 << n_bits
        self.ALL = (1 << self.P) - 1

    def column(self, j: int) -> int:
        """Bitset of 'bit j of the vector index p' over p in [0, 2^n)."""
        out = 0
        block = 1 << j
        period = block << 1
        ones = ((1 << block) - 1) << block     # within one period: low half 0, high half 1
        p = 0
        while p < self.P:
            out |= ones << p
            p += period
        return out & self.ALL


def _ext(bits: List[int], w: int, fill: int = 0) -> List[int]:
    return [bits[i] if i < len(bits) else fill for i in range(w)]


def evaluate(design, fault: Optional[Tuple[int, int, int]] = None) -> Tuple[List[List[int]], Bitsets]:
    """Bitsets of every net bit, nodes evaluated in index order (generator order is
    topological). fault = (net, bit, value) or None."""
    I = design.n_in
    assert design.n_reg == 0, "combinational designs only"
    n_bits = int(np.sum(design.input_widths.astype(np.int64)))
    bs = Bitsets(n_bits)
    ALL = bs.ALL
    nets: List[List[int]] = []

    def force(net_id: int, bits: List[int]) -> List[int]:
        if fault is not None and fault[0] == net_id:
            bits = list(bits)
            if fault[2] >= 2:              # a flip in every vector (transient model)
                bits[fault[1]] ^= ALL
            else:
                bits[fault[1]] = ALL if fault[2] else 0
        return bits

    j = 0
    for i in range(I):
        w = int(design.input_widths[i])
        nets.append(force(i, [bs.column(j + k) for k in range(w)]))
        j += w
    for n in range(design.n_node):
        op = int(design.node_op[n])
        w = int(design.node_w[n])
        A = nets[int(design.node_a[n])] if op != CONST else []
        B = nets[int(design.node_b[n])] if op not in (CONST, NOT, SHL, SHR, SLICE) else []
        C = nets[int(design.node_c[n])] if op == MUX2 else []
        k = int(design.node_imm[n])
        if op == AND:
            a, b = _ext(A, w), _ext(B, w)
            out = [x & y for x, y in zip(a, b)]
        elif op == OR:
            a, b = _ext(A, w), _ext(B, w)
            out = [x | y for x, y in zip(a, b)]
        elif op == XOR:
            a, b = _ext(A, w), _ext(B, w)
            out = [x ^ y for x, y in zip(a, b)]
        elif op == NOT:
            out = [ALL ^ x for x in _ext(A, w)]
        elif op in (ADD, SUB):
            a = _ext(A, w)
            b = _ext(B, w)
            if op == SUB:                      # a - b = a + ~b + 1 (two's complement)
                b = [ALL ^ x for x in b]
                carry = ALL
            else:
                carry = 0
            out = []
            for x, y in zip(a, b):
                out.append(x ^ y ^ carry)
                carry = (x & y) | (carry & (x ^ y))
        elif op == MUX2:
            sel = 0
            for x in A:
                sel |= x
            b, c = _ext(B, w), _ext(C, w)
            out = [(sel & x) | ((ALL ^ sel) & y) for x, y in zip(b, c)]
        elif op == EQ:
            m = max(len(A), len(B))
            eq = ALL
            for x, y in zip(_ext(A, m), _ext(B, m)):
                eq &= ALL ^ (x ^ y)
            out = [eq]
        elif op == LT:
            m = max(len(A), len(B))
            lt = 0                             # borrow of a - b, LSB to MSB
            for x, y in zip(_ext(A, m), _ext(B, m)):
                lt = ((ALL ^ x) & y) | ((ALL ^ (x ^ y)) & lt)
            out = [lt]
        elif op == SHL:
            out = [(A[i - k] if 0 <= i - k < len(A) else 0) for i in range(w)]
        elif op in (SHR, SLICE):
            out = [(A[i + k] if i + k < len(A) else 0) for i in range(w)]
        elif op == CONCAT:
            wb = len(B)
            out = [(B[i] if i < wb else (A[i - wb] if i - wb < len(A) else 0)) for i in range(w)]
        elif op == CONST:
            out = [ALL if (k >> i) & 1 else 0 for i in range(w)]
        else:
            raise ValueError(op)
        nets.append(force(I + n, out[:w]))
    return nets, bs


def brute_force(design, faults) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(detected, first vector index, first port) of every fault under the stimulus that
    enumerates all input vectors in counting order."""
    good, bs = evaluate(design)
    F = len(faults)
    det = np.zeros(F, np.uint8)
    cyc = np.full(F, -1, np.int32)
    port = np.full(F, -1, np.int32)
    outs = [int(o) for o in design.outputs]
    for f in range(F):
        bad, _ = evaluate(design, (int(faults.net[f]), int(faults.bit[f]), int(faults.val[f])))
        per_port = []
        anydiff = 0
        for o in outs:
            d = 0
            for x, y in zip(good[o], bad[o]):
                d |= x ^ y
            per_port.append(d)
            anydiff |= d
        if anydiff:
            p = (anydiff & -anydiff).bit_length() - 1
            det[f] = 1
            cyc[f] = p
            port[f] = next(i for i, d in enumerate(per_port) if (d >> p) & 1)
    return det, cyc, port


def exhaustive_stimulus(design) -> np.ndarray:
    """[2^n, I] stimulus: cycle p applies vector p, input i taking its slice of p's bits."""
    widths = [int(w) for w in design.input_widths]
    n = sum(widths)
    p = np.arange(1 << n, dtype=np.uint64)
    cols = []
    j = 0
    for w in widths:
        cols.append((p >> np.uint64(j)) & np.uint64((1 << w) - 1))
        j += w
    return np.ascontiguousarray(np.stack(cols, axis=1).astype(np.uint64))


def brute_force_ex(design, faults) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """(detected, first vector, first port, vectors with a differing port) under the
    exhaustive stimulus, for the general fault list: kinds 0/1 stuck-at, kind 3 (SET) a
    flip in the single vector faults.cycle[f]; net ids n_net + o are output-port faults,
    whose force applies to what port o observes only. For a combinational design the
    machines of different vectors are independent, so an SET at vector c is detected iff
    the flip, applied to every vector at once, changes an output in vector c."""
    good, bs = evaluate(design)
    F = len(faults)
    det = np.zeros(F, np.uint8)
    cyc = np.full(F, -1, np.int32)
    port = np.full(F, -1, np.int32)
    count = np.zeros(F, np.uint32)
    outs = [int(o) for o in design.outputs]
    n_net = design.n_net
    for f in range(F):
        net, b, kind = int(faults.net[f]), int(faults.bit[f]), int(faults.val[f])
        per_port = []
        if net >= n_net:        # port fault: the other ports see the good machine
            o = net - n_net
            for q, on in enumerate(outs):
                d = 0
                if q == o:
                    g = good[on][b]
                    d = g ^ (bs.ALL ^ g if kind >= 2 else (bs.ALL if kind else 0))
                per_port.append(d)
        else:
            bad, _ = evaluate(design, (net, b, kind))
            for on in outs:
                d = 0
                for x, y in zip(good[on], bad[on]):
                    d |= x ^ y
                per_port.append(d)
        anydiff = 0
        for d in per_port:
            anydiff |= d
        if kind >= 2:           # only the flip's own vector can differ
            c = int(faults.cycle[f])
            anydiff &= (1 << c) if c < bs.P else 0
            per_port = [d & anydiff for d in per_port]
        count[f] = bin(anydiff).count("1")
        if anydiff:
            p0 = (anydiff & -anydiff).bit_length() - 1
            det[f] = 1
            cyc[f] = p0
            port[f] = next(i for i, d in enumerate(per_port) if (d >> p0) & 1)
    return det, cyc, port, count
