"""Pins of the load-predictor and feature oracle (oracle/mlp.py), independent of it:

* BF16 rounding against float32 values whose BF16 neighbours are known by construction;
* the gradient against central finite differences of the loss (float64);
* a network whose pre-activations are all positive is affine, so its output equals the
  product of its weight matrices applied to the input (closed form);
* the features of the hand-checkable 4-bit counter, derived by hand.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2508_16376_gb300 import synth
import oracle


def _rand_bits(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return mlp.f64_to_bf16_bits(rng.normal(0, scale, mlp.N_PARAMS))


def test_bf16_rounding_known_values():
    # 1 + 2^-8 lies exactly between BF16 1.0 and 1 + 2^-7: ties go to even (1.0)
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1.0 + 2 ** -9], np.float64)
    bits = mlp.f64_to_bf16_bits(vals)
    back = mlp.bf16_bits_to_f64(bits)
    assert list(back) == [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 0.0, 1.0]
    assert bits[0] == 0x3F80 and bits[3] == 0xC020


def test_gradient_matches_finite_differences():
    w = _rand_bits(1)
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (7, 5))
    t = rng.normal(0, 1, 7)
    loss, g = mlp.loss_grad(w, X, t)
    p = mlp.bf16_bits_to_f64(w)

    def L(q):
        # loss at arbitrary float64 parameters (same definitions, no BF16 rounding)
        W1, b1, W2, b2, w3, b3 = mlp.unpack(q)
        h1 = np.maximum(X @ W1 + b1, 0)
        h2 = np.maximum(h1 @ W2 + b2, 0)
        y = h2 @ w3 + b3
        return np.mean((y - t) ** 2)

    assert abs(L(p) - loss) < 1e-12
    idx = list(range(0, mlp.N_PARAMS, 97)) + [mlp.OFF_B3, mlp.OFF_W3 + 3, mlp.OFF_B1 + 5]
    h = 1e-6
    for i in idx:
        q1, q2 = p.copy(), p.copy()
        q1[i] += h
        q2[i] -= h
        fd = (L(q1) - L(q2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_all_positive_network_is_affine():
    rng = np.random.default_rng(3)
    p = np.abs(rng.normal(0, 0.2, mlp.N_PARAMS)) + 0.01     # every weight and bias > 0
    w = mlp.f64_to_bf16_bits(p)
    q = mlp.bf16_bits_to_f64(w)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(q)
    X = rng.uniform(0, 1, (11, 5))
    y, _ = mlp.forward(w, X)
    expected = X @ (W1 @ W2 @ w3) + (b1 @ W2 @ w3 + b2 @ w3 + b3)
    assert np.allclose(y, expected, rtol=1e-12, atol=1e-12)


def test_counter_features_by_hand():
    """Counter: nets 0 input, 1 Q, 2 c=CONST, 3 s=ADD(Q,c), 4 x=XOR(Q,c); output = Q.
    Consumers: Q -> {s, x}, c -> {s, x}, s -> {} (only the register), x -> {}.
    Cone estimates: s = x = 1, Q = c = 1 + 1 + 1 = 3. Levels: c 0, s 1, x 1 -> n_levels 2.
    Register depth: Q is the output (0); s feeds Q's register (1); c feeds s (1); x reaches
    nothing (16). Toggles over t = 1..19 of: Q bit 0 (Q_t = t mod 16): every cycle, 19;
    Q bit 3: at t = 8 and 16, 2; c: never; s bit 2 (s_t = (t+1) mod 16): when t+1 is a
    multiple of 4, t = 3, 7, 11, 15, 19, 5; x bit 1 (x_t = t XOR 1, bit 1 of t): at
    t = 2, 4, ..., 18, 9."""
    d = synth.counter4()
    T = 20
    stim = np.zeros((T, 1), np.uint64)
    _, trace = oracle.good_run(d, stim, with_trace=True)
    f = synth.Faults(np.array([1, 1, 2, 3, 4], np.uint32), np.array([0, 3, 0, 2, 1], np.uint8),
                     np.zeros(5, np.uint8))
    X = mlp.features(d, trace, f)
    exp = np.array([
        [np.log2(3) / 20, 0.0, 0.0, 4 / 64, 19 / 19],
        [np.log2(3) / 20, 0.0, 0.0, 4 / 64, 2 / 19],
        [np.log2(3) / 20, 1 / 2, 1 / 16, 4 / 64, 0.0],
        [0.0, 2 / 2, 1 / 16, 4 / 64, 5 / 19],
        [0.0, 2 / 2, 1.0, 4 / 64, 9 / 19],
    ])
    assert np.allclose(X, exp, atol=1e-12), X


def test_toggle_rate_uses_the_first_256_cycles():
    """Counter over T = 300 cycles: the toggle rate counts changes over t = 1..255 only (the
    prefix a campaign has when it orders its first window). Q bit 0 changes every cycle:
    255 / 255. Q bit 3 (Q_t = t mod 16) changes when t is a multiple of 8: 31 times in
    1..255 -> 31 / 255 (over the whole stimulus it would be 37 / 299). s bit 0
    (s_t = (t+1) mod 16) changes every cycle: 1."""
    d = synth.counter4()
    stim = np.zeros((300, 1), np.uint64)
    _, trace = oracle.good_run(d, stim, with_trace=True)
    f = synth.Faults(np.array([1, 1, 3], np.uint32), np.array([0, 3, 0], np.uint8), np.zeros(3, np.uint8))
    X = mlp.features(d, trace, f)
    assert np.allclose(X[:, 4], [1.0, 31 / 255, 1.0], atol=1e-12), X[:, 4]
