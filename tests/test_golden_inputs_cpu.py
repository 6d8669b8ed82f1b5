"""The stored full-size oracle results (tests/golden/fullsize/) still describe the inputs the
generator builds today: every stored design's fingerprint equals the fingerprint of the
design, stimulus and fault list synth produces for it, the stored fault indices are in range,
the results are well formed (detected faults carry a cycle and a port inside the design's
ranges, undetected ones -1/-1), and the stratified rule's FSM-bit faults are all stored."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fullsize_golden as golden  # noqa: E402

from paper_2508_16376_gb300 import synth  # noqa: E402


def _inputs(name):
    if name == "medium":
        return [synth.workload("medium")]
    if name == "large":
        return [synth.workload("large")]
    return synth.batch_workload()


@pytest.mark.parametrize("name", ["medium", "large", "batch"])
def test_stored_results_match_todays_inputs(name):
    stored = golden.load(name)
    assert stored, name
    parts = _inputs(name)
    for di, (fp, idx, det, cyc, port) in stored.items():
        d, stim, f = parts[di]
        assert golden.fingerprint(d, stim, f) == fp, (name, di)
        assert len(idx) and idx.max() < len(f) and np.all(np.diff(idx) > 0)
        T = stim.shape[0]
        hit = det == 1
        assert set(np.unique(det)) <= {0, 1}
        assert np.all((cyc[hit] >= 0) & (cyc[hit] < T)) and np.all((port[hit] >= 0) & (port[hit] < d.n_out))
        assert np.all(cyc[~hit] == -1) and np.all(port[~hit] == -1)
        if name != "medium":   # every sampled fault on an FSM state bit is stored
            ctrl = np.nonzero(np.isin(f.net, d.control_nets))[0]
            assert np.isin(ctrl, idx).all(), (name, di)
        else:
            assert np.array_equal(idx, np.arange(len(f)))
