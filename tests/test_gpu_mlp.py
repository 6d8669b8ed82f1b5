"""GPU parity of the load predictor and its features (through the C-ABI) against the
float64 oracle in oracle/mlp.py, and the rule that the predictor never changes a result.

Tolerances: features are single-precision values of exactly defined quantities (1e-6
absolute). The forward pass accumulates in FP32 where the oracle uses float64 on the same
BF16 weights: 64-term dot products of O(1) terms give relative errors of order 1e-6, so
1e-4 relative (1e-5 absolute) is loose. Gradients sum FP32 atomics in an unspecified
order: 1e-3 of the largest gradient entry."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2508_16376_gb300 import synth, rtlfs
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _weights(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return mlp.f64_to_bf16_bits(rng.normal(0, scale, mlp.N_PARAMS))


@pytest.mark.parametrize("maker,T,F", [(lambda: synth.tiny_design(1), 100, 2000),
                                       (lambda: synth.gen_datapath_fsm(8, 3000, 300, 16, 16, [8], 0.8, 12, 64), 257, 3000)])
def test_features_match_oracle(maker, T, F):
    d = maker()
    stim = synth.stimulus(d, T, 3, 0.1)
    f = synth.sample_faults(d, F, 3)
    _, trace = oracle.good_run(d, stim, with_trace=True)
    exp = mlp.features(d, trace, f)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        X = rtlfs.rtlfs_features(sim.ctx, 0, F)
    assert np.allclose(X, exp, atol=1e-6), np.abs(X - exp).max(axis=0)


def test_forward_and_gradient_match_oracle():
    w = _weights(5)
    rng = np.random.default_rng(6)
    n = 1000                                  # spans several 64-sample tiles, ragged tail
    X = rng.uniform(0, 1, (n, 5)).astype(np.float32)
    t = rng.normal(2, 1, n).astype(np.float32)
    ctx = rtlfs.rtlfs_create(0)
    try:
        rtlfs.rtlfs_mlp_set_weights(ctx, w)
        assert np.array_equal(rtlfs.rtlfs_mlp_get_weights(ctx), w)
        y = rtlfs.rtlfs_mlp_forward(ctx, X)
        ey, _ = mlp.forward(w, X.astype(np.float64))
        assert np.allclose(y, ey, rtol=1e-4, atol=1e-5)
        loss, g = rtlfs.rtlfs_mlp_grad(ctx, X, t)
        eloss, eg = mlp.loss_grad(w, X.astype(np.float64), t.astype(np.float64))
        assert abs(loss - eloss) <= 1e-4 * abs(eloss) + 1e-6
        assert np.abs(g - eg).max() <= 1e-3 * np.abs(eg).max(), np.abs(g - eg).max()
    finally:
        rtlfs.rtlfs_destroy(ctx)


def test_training_reduces_loss():
    rng = np.random.default_rng(7)
    n = 4096
    X = rng.uniform(0, 1, (n, 5)).astype(np.float32)
    t = (3 * X[:, 0] + np.sin(4 * X[:, 4]) + X[:, 1] * X[:, 2]).astype(np.float32)
    w = _weights(8, 0.1)
    ctx = rtlfs.rtlfs_create(0)
    try:
        rtlfs.rtlfs_mlp_set_weights(ctx, w)
        l0, _ = rtlfs.rtlfs_mlp_grad(ctx, X, t)
        l1 = rtlfs.rtlfs_mlp_train(ctx, X, t, epochs=30, batch=256, lr=3e-3)
        l2, _ = rtlfs.rtlfs_mlp_grad(ctx, X, t)
        assert l2 < 0.1 * l0, (l0, l1, l2)
        # the trained BF16 weights reproduce the reported loss in the oracle
        wt = rtlfs.rtlfs_mlp_get_weights(ctx)
        el, _ = mlp.loss_grad(wt, X.astype(np.float64), t.astype(np.float64))
        assert abs(el - l2) <= 1e-3 * el + 1e-6
    finally:
        rtlfs.rtlfs_destroy(ctx)


@pytest.mark.parametrize("seed", [1, 2])
def test_predictor_never_changes_results(seed):
    """Garbage weights, trained-looking weights, heuristic and plain schedules, with and
    without heavy pre-assignment: identical results, equal to the oracle's."""
    d = synth.gen_datapath_fsm(30 + seed, 2500, 250, 16, 16, [8], 0.8, 12, 64)
    stim = synth.stimulus(d, 300, seed, 0.1)
    f = synth.sample_faults(d, 3000, seed)
    exp = oracle.fault_sim(d, stim, f, threads=16)
    with Simulator(0) as sim:
        sim.add(d, stim, f)
        for w in (_weights(seed, 5.0), _weights(seed + 10, 0.05)):
            rtlfs.rtlfs_mlp_set_weights(sim.ctx, w)
            for hf in (0.0, 0.05, 0.5):
                res, _ = sim.run(scheduler=rtlfs.SCHED_MLP, heavy_frac=hf)
                got = split(res[0])
                for a, b in zip(got, exp):
                    assert np.array_equal(a, b)
        for sch in (rtlfs.SCHED_PLAIN, rtlfs.SCHED_HEURISTIC):
            res, _ = sim.run(scheduler=sch, heavy_frac=0.1)
            for a, b in zip(split(res[0]), exp):
                assert np.array_equal(a, b)
