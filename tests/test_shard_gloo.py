"""The multi-rank path on CPU: world_size-2 gloo process groups shard a fault list by
predicted load, each rank simulates its shard (the CPU oracle stands in for a rank's GPU),
and the gathered results equal the single-process run. Also the shard balance."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_16376_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 100, 101)
    f = synth.fault_universe(d)
    pred = np.random.default_rng(0).uniform(0, 10, len(f))
    det, cyc, port_ = shard.run_sharded(f, pred, lambda sub: oracle.fault_sim(d, stim, sub, threads=2))
    if rank == 0:
        np.savez(out_path, det=det, cyc=cyc, port=port_)
    dist.barrier()
    dist.destroy_process_group()


def _campaign_worker(rank, world, port, out_path):
    """bench.py's rank path on two designs: LPT shards of each design's list from the same
    predicted loads, this rank's shards simulated (the oracle stands in for the GPU), and
    gather_results assembling full-length results on every rank."""
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = _two_designs()
    pred = [np.random.default_rng(7 + i).uniform(0, 10, len(f)) for i, (_, _, f) in enumerate(parts)]
    mine = [shard.lpt_shards(p, world)[rank] for p in pred]
    res = [np.stack(oracle.fault_sim(d, s, f.take(m), threads=2)).astype(np.int64)
           for (d, s, f), m in zip(parts, mine)]
    full = shard.gather_results(res, mine, [len(f) for _, _, f in parts])
    np.savez(out_path + f".{rank}.npz", *full)
    dist.barrier()
    dist.destroy_process_group()


def _two_designs():
    out = []
    for seed in (1, 2):
        d = synth.tiny_design(seed)
        out.append((d, synth.stimulus(d, 80, 100 + seed), synth.sample_faults(d, 1500, seed)))
    return out


def test_two_rank_campaign_shards_gather_on_every_rank(tmp_path):
    import oracle
    oracle.build()
    out = str(tmp_path / "camp")
    mp.start_processes(_campaign_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        r = np.load(out + f".{rank}.npz")
        for i, (d, s, f) in enumerate(_two_designs()):
            exp = np.stack(oracle.fault_sim(d, s, f, threads=4))
            assert np.array_equal(r[f"arr_{i}"], exp)


def test_two_rank_gloo_gather_equals_single_run(tmp_path):
    import oracle
    oracle.build()
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    d = synth.tiny_design(1)
    stim = synth.stimulus(d, 100, 101)
    exp = oracle.fault_sim(d, stim, synth.fault_universe(d), threads=4)
    assert np.array_equal(r["det"], exp[0])
    assert np.array_equal(r["cyc"], exp[1])
    assert np.array_equal(r["port"], exp[2])


@pytest.mark.parametrize("world", [2, 3, 8])
def test_lpt_shards_partition_and_balance(world):
    rng = np.random.default_rng(world)
    pred = np.exp(rng.normal(0, 2, 5000))          # heavy-tailed loads
    parts = shard.lpt_shards(pred, world)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(5000))
    # LPT is within 4/3 of optimal; with many small items it is near 1
    assert shard.shard_imbalance(pred, parts) < 1.05


def test_single_process_path_without_group():
    calls = []
    res = shard.run_sharded(synth.Faults(np.zeros(3, np.uint32), np.zeros(3, np.uint8), np.zeros(3, np.uint8)),
                            np.ones(3), lambda sub: calls.append(len(sub)) or (1, 2, 3))
    assert calls == [3] and res == (1, 2, 3)
