"""Load-predictor and feature oracle -- TEST INFRASTRUCTURE ONLY (numpy, float64).

The network is the plain definition of a 5-64-64-1 multilayer perceptron with ReLU hidden
layers and a linear output, evaluated in float64 on the BF16 parameter values it is given
(bit patterns, so both sides see identical weights), with the mean squared error and its
gradient by the chain rule written out layer by layer. Parameter layout: W1[5][64], b1[64],
W2[64][64], b2[64], w3[64], b3.

The features are the plain definitions of the five per-fault inputs, computed from the
design arrays and the oracle's good trace: static fan-out cone estimate, topological
level, register depth to the outputs, width, and toggle rate of the site bit over the
first min(T, TOGGLE_CYCLES) cycles (the prefix a campaign has simulated when it orders its
first cycle window).
"""
from __future__ import annotations

from collections import deque

import numpy as np

IN, H = 5, 64
TOGGLE_CYCLES = 256
OFF_B1 = IN * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
N_PARAMS = OFF_B3 + 1


def bf16_bits_to_f64(w: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) -> float64 values (exact)."""
    return (np.asarray(w, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def f64_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to BF16 (round to nearest, ties to even) -> uint16 bit patterns.
    Implements the published BF16 format: the upper 16 bits of the IEEE binary32 value,
    rounded on the 16 dropped bits."""
    f = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = (f + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def unpack(p: np.ndarray):
    W1 = p[:OFF_B1].reshape(IN, H)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(H, H)
    b2 = p[OFF_B2:OFF_W3]
    w3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def forward(w_bits: np.ndarray, X: np.ndarray):
    """Returns y[n] and the intermediate pre-activations (a1, a2) and activations."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16_bits_to_f64(w_bits))
    X = np.asarray(X, np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (a1, h1, a2, h2)


def loss_grad(w_bits: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error over the samples and its gradient w.r.t. every parameter."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16_bits_to_f64(w_bits))
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    n = X.shape[0]
    y, (a1, h1, a2, h2) = forward(w_bits, X)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n                       # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)       # dL/da2
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (a1 > 0)            # dL/da1
    g_W1 = X.T @ d1
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


# ---- features --------------------------------------------------------------------------

_NOPS = {13: 0, 3: 1, 9: 1, 10: 1, 11: 1, 6: 3}


def _operands(design, i):
    k = _NOPS.get(int(design.node_op[i]), 2)
    return [int(design.node_a[i]), int(design.node_b[i]), int(design.node_c[i])][:k]


def features(design, trace: np.ndarray, faults) -> np.ndarray:
    """[F, 5] float64 features, from their definitions."""
    I, R, N = design.n_in, design.n_reg, design.n_node
    base = I + R
    nn = design.n_net
    ops = [_operands(design, i) for i in range(N)]
    # topological level: longest chain of node operands (0 when a node reads no node)
    level = {}

    def lev(i):
        stack = [i]
        while stack:
            j = stack[-1]
            if j in level:
                stack.pop()
                continue
            pend = [x - base for x in ops[j] if x >= base and (x - base) not in level]
            if pend:
                stack.extend(pend)
                continue
            level[j] = max([level[x - base] + 1 for x in ops[j] if x >= base], default=0)
            stack.pop()
        return level[i]

    for i in range(N):
        lev(i)
    n_levels = (max(level.values()) + 1) if N else 0
    # consumers of each net (distinct nodes), cone estimate = 1 + sum over consumers
    cons = [[] for _ in range(nn)]
    for i in range(N):
        for x in sorted(set(ops[i])):
            cons[x].append(base + i)
    cone = np.ones(nn, np.float64)
    order = sorted(range(N), key=lambda i: -level[i])     # consumers before producers
    for i in order:
        cone[base + i] = min(1.0 + sum(cone[c] for c in cons[base + i]), 1e9)
    for e in range(base):
        cone[e] = min(1.0 + sum(cone[c] for c in cons[e]), 1e9)
    # register depth to the outputs: fewest register stages on a path to an output
    depth = np.full(nn, np.inf)
    dq = deque()
    for o in design.outputs:
        depth[int(o)] = 0
        dq.appendleft(int(o))
    while dq:
        y = dq.popleft()
        d = depth[y]
        if y >= base:
            for x in ops[y - base]:
                if depth[x] > d:
                    depth[x] = d
                    dq.appendleft(x)
        elif y >= I:
            x = int(design.reg_d[y - I])
            if depth[x] > d + 1:
                depth[x] = d + 1
                dq.append(x)
    widths = design.net_widths().astype(np.float64)
    T = min(trace.shape[0], TOGGLE_CYCLES)
    F = len(faults)
    X = np.zeros((F, 5), np.float64)
    for f in range(F):
        s, b = int(faults.net[f]), int(faults.bit[f])
        X[f, 0] = min(np.log2(cone[s]) / 20.0, 1.5)
        X[f, 1] = 0.0 if s < base else (level[s - base] + 1) / max(n_levels, 1)
        X[f, 2] = min(depth[s], 16) / 16.0
        X[f, 3] = widths[s] / 64.0
        bits = (trace[:T, s] >> np.uint64(b)) & np.uint64(1)
        X[f, 4] = (np.count_nonzero(bits[1:] != bits[:-1]) / (T - 1)) if T > 1 else 0.0
    return X
