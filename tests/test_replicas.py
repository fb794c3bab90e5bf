"""Multi-rank plumbing of bench.py on CPU: world_size 2 over gloo.

Replicas share no data of the method; the ranks meet only to agree on timing. These
tests run the same helpers bench.py uses under torchrun (RankSync, replica_temperatures)
in two gloo processes.
"""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sync = bench.RankSync(dist, device="cpu")
    temps1 = bench.replica_temperatures(1, rank, world)
    temps4 = bench.replica_temperatures(4, rank, world)
    sync.barrier()
    flops = 1e12 * (rank + 1)           # rank r "did" (r+1) TFLOP
    ms = 100.0 * (rank + 1)             # in (r+1) * 100 ms
    value, ms_max = sync.throughput(flops, ms)
    out[rank] = (temps1, temps4, value, ms_max, sync.max(rank), sync.sum(1.0))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    # distinct, non-overlapping temperatures
    assert r0[0] != r1[0]
    assert set(r0[1]).isdisjoint(r1[1]) and len(r0[1]) == len(r1[1]) == 4
    assert min(r1[1]) > max(r0[1])
    # whole-job throughput = all flops / slowest rank: 3 TFLOP / 0.2 s = 15 TFLOP/s, on every rank
    for r in (r0, r1):
        assert r[2] == pytest.approx(15.0)
        assert r[3] == pytest.approx(200.0)
        assert r[4] == pytest.approx(1.0) and r[5] == pytest.approx(2.0)


def test_single_rank_needs_no_process_group():
    import bench
    sync = bench.RankSync(None)
    assert sync.throughput(2e12, 500.0) == (pytest.approx(4.0), 500.0)
    assert bench.replica_temperatures(1, 0, 1) == [6.65]
