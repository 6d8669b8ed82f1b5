"""GPU test of rtlfs_fault_sim_static, the allocation-free entry point.

It is meant for callers that cannot obtain device memory from cudaMalloc where they run --
a process whose GPU memory belongs to another allocator (here torch's caching pool plays
that allocator), or a latency-critical path that cannot take an allocation: they pass
their own device buffers for the faults and the results, and the library takes its
scratch from a fixed array in its own image. The test checks, on two calls in a row, that
the results equal those of the existing entry point rtlfs_run and of the oracle on the
same faults (the tolerance every result test in this suite uses: bit-exact), that the
device's free memory does not change across the calls, and that output-port faults are
refused. It lives in a file collected last and builds what it needs itself, so it passes
alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16376_gb300 import rtlfs, synth
from paper_2508_16376_gb300.rtlfs import Simulator, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_16376_gb300 import build
    build.build()
    oracle.build()


def _device_bytes(arr: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).copy()).cuda()


CASES = {
    # all 6,054 faults of the tiny design, input nets included, one wave
    "tiny_all_with_inputs": (lambda: synth.tiny_design(1), 100, None, {}),
    # an FSM-steered datapath, several waves; the reference campaign runs in windows of
    # 256 cycles, so the good trace the static call reads was written window by window
    "fsm_windowed": (lambda: synth.gen_datapath_fsm(8, 3000, 300, 16, 16, [8], 0.8, 12, 64), 600, 3000,
                     {"window": 256, "light_cap": 1}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_entry_point_matches_rtlfs_run_and_oracle(case):
    import torch
    maker, T, F, run_opts = CASES[case]
    d = maker()
    stim = synth.stimulus(d, T, 4, 0.1)
    faults = synth.fault_universe(d, include_inputs=True) if F is None else synth.sample_faults(d, F, 4)
    n = len(faults)
    odet, ocyc, oport = oracle.fault_sim(d, stim, faults, threads=16)
    with Simulator(0) as sim:
        sim.add(d, stim, faults)
        ref, _ = sim.run(**run_opts)                 # existing entry point; leaves the good trace
        exp = split(ref[0])
        for a, b in zip(exp, (odet, ocyc, oport)):
            assert np.array_equal(a, b)
        fa = _device_bytes(rtlfs.fault_array(faults))
        out = torch.empty(n * rtlfs.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        free = []
        for call in range(3):                        # calls in a row share the static scratch
            out.fill_(0xA5)                          # stale bytes must not survive
            torch.cuda.synchronize()
            before = torch.cuda.mem_get_info()[0]
            rc = rtlfs.rtlfs_fault_sim_static(sim.ctx, 0, fa.data_ptr(), n, out.data_ptr(), stream)
            torch.cuda.synchronize()
            free.append((before, torch.cuda.mem_get_info()[0]))
            assert rc == rtlfs.RTLFS_OK, rtlfs.rtlfs_last_error(sim.ctx)
            got = out.cpu().numpy().view(rtlfs.RESULT_DTYPE)
            for a, b in zip(split(got), exp):
                assert np.array_equal(a, b), f"call {call}"
    # the first call on a device may load the library's module (its static array); after
    # that no call changes the device's free memory
    for before, after in free[1:]:
        assert before == after, free


def test_static_entry_point_refuses_port_faults_and_bad_bits():
    import torch
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 50, 4)
    good = synth.sample_faults(d, 20, 4)
    bad = synth.Faults(np.array([d.n_net, d.n_net + 1, 10], np.uint32),   # two ports, one bit past the width
                       np.array([0, 0, 63], np.uint8), np.array([0, 1, 1], np.uint8))
    f = synth.Faults.concat([good, bad])
    with Simulator(0) as sim:
        sim.add(d, stim, good)
        ref, _ = sim.run()
        fa = _device_bytes(rtlfs.fault_array(f))
        out = torch.empty(len(f) * rtlfs.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        rc = rtlfs.rtlfs_fault_sim_static(sim.ctx, 0, fa.data_ptr(), len(f), out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
        assert rc == rtlfs.RTLFS_E_ARG
        got = out.cpu().numpy().view(rtlfs.RESULT_DTYPE)
    assert list(got["detected"][-3:]) == [254, 254, 254]
    for a, b in zip(split(got[:20]), split(ref[0])):
        assert np.array_equal(a, b)


def test_static_entry_point_needs_a_current_good_trace():
    d = synth.tiny_design(2)
    stim = synth.stimulus(d, 20, 2)
    faults = synth.sample_faults(d, 10, 2)
    with Simulator(0) as sim:
        sim.add(d, stim, faults)                    # no run yet: no good trace
        rc = rtlfs.rtlfs_fault_sim_static(sim.ctx, 0, 0, 0, 0, 0)
        assert rc == rtlfs.RTLFS_E_STATE
