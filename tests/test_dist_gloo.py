"""Multi-process paths of bench.py on CPU (gloo, world size 2).

One apply does not shard (replicas only): each rank times its own replica,
the step time is the maximum over ranks, and the throughput sums the units
of all ranks.  The batch of uneven instances shards by instance with no
exchange: every instance goes to exactly one rank, the work is balanced,
and the throughput is the sum of the ranks' own units over the slowest
rank's time.  The tests run two gloo ranks and check both reductions.
"""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    dist.barrier()
    ms, value = bench.aggregate(local_ms, 1000, 10, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == pytest.approx(15.0)                 # max(100, 150) / 10 steps
        assert value == pytest.approx(2 * 1000 / 15e-3)  # both replicas' units / slowest time


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate(50.0, 100, 5)
    assert ms == 10.0 and value == pytest.approx(100 / 10e-3)


def _worker_sharded(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    insts = synth.batched_instances(32, 1)
    work = [w.N * w.nrhs for w in insts]
    mine = bench.shard_instances(work, world, rank)
    units = sum(2 * insts[i].N * insts[i].nrhs for i in mine)
    ms, value = bench.aggregate_sharded(100.0 + 20.0 * rank, units, 10, dist, torch.device("cpu"))
    q.put((rank, mine, units, ms, value))
    dist.destroy_process_group()


def test_two_rank_instance_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    sys.path.insert(0, ROOT)
    import synth
    insts = synth.batched_instances(32, 1)
    got = sorted(res[0][1] + res[1][1])
    assert got == list(range(len(insts)))                    # each instance exactly once
    w0 = sum(insts[i].N * insts[i].nrhs for i in res[0][1])
    w1 = sum(insts[i].N * insts[i].nrhs for i in res[1][1])
    assert abs(w0 - w1) <= max(w.N * w.nrhs for w in insts)  # balanced to within one instance
    total = sum(2 * w.N * w.nrhs for w in insts)
    for rank, mine, units, ms, value in res:
        assert ms == pytest.approx(12.0)                      # max(100, 120) / 10 steps
        assert value == pytest.approx(total / 12e-3)          # the whole batch / slowest time
