"""GPU test of rtlfs_fault_sim_static, the allocation-free entry point.

It is meant for callers that cannot allocate device memory where they run (inside a
stream capture, on latency-critical paths, or under another framework's allocator): they
pass their own device buffers for the faults and the results, and the library takes its
scratch from a fixed array in its own image. This test plays such a caller with buffers
from torch's allocator, and checks that two calls in a row return exactly the results of
the existing entry point rtlfs_run on the same faults (the tolerance every result test in
this suite uses: bit-exact). It lives in a file collected last, and builds what it needs
itself, so it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2508_16376_gb300 import rtlfs, synth
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()


def _device_bytes(arr: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).copy()).cuda()


@pytest.mark.parametrize("maker,T,F", [
    (lambda: synth.tiny_design(1), 100, None),                       # all 5,926 faults, one wave
    (lambda: synth.gen_datapath_fsm(8, 3000, 300, 16, 16, [8], 0.8, 12, 64), 300, 3000),  # several waves
])
def test_static_entry_point_matches_rtlfs_run(maker, T, F):
    import torch
    d = maker()
    stim = synth.stimulus(d, T, 4, 0.1)
    faults = synth.fault_universe(d) if F is None else synth.sample_faults(d, F, 4)
    n = len(faults)
    with Simulator(0) as sim:
        sim.add(d, stim, faults)
        ref, _ = sim.run()                          # existing entry point; also leaves the good trace
        exp = split(ref[0])
        fa = _device_bytes(rtlfs.fault_array(faults))
        out = torch.empty(n * rtlfs.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):                      # two calls in a row share the static scratch
            out.fill_(0xA5)                         # stale bytes must not survive
            rc = rtlfs.rtlfs_fault_sim_static(sim.ctx, 0, fa.data_ptr(), n, out.data_ptr(), stream)
            assert rc == rtlfs.RTLFS_OK, rtlfs.rtlfs_last_error(sim.ctx)
            got = out.cpu().numpy().view(rtlfs.RESULT_DTYPE)
            for a, b in zip(split(got), exp):
                assert np.array_equal(a, b), f"call {call}"


def test_static_entry_point_needs_a_current_good_trace():
    d = synth.tiny_design(2)
    stim = synth.stimulus(d, 20, 2)
    faults = synth.sample_faults(d, 10, 2)
    with Simulator(0) as sim:
        sim.add(d, stim, faults)                    # no run yet: no good trace
        rc = rtlfs.rtlfs_fault_sim_static(sim.ctx, 0, 0, 0, 0, 0)
        assert rc == rtlfs.RTLFS_E_STATE
