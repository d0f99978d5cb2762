"""The multi-process path of bench.py on CPU (gloo, world size 2): ranks take
disjoint blocks of instances, the timing reduction takes the slowest rank,
and the whole-job rate counts every rank's instances. No GPU is used."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, n = bench.replica_instances(rank, world, 608)
        ms = 100.0 + 25.0 * rank  # rank 1 is the slowest
        ms_max = bench.max_over_ranks(ms, world)
        out.put((rank, first, n, ms_max, bench.whole_job_rate(world, n, ms_max)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_partition_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, f0, n0, m0, v0), (r1, f1, n1, m1, v1) = res
    assert (f0, n0, f1, n1) == (0, 608, 608, 608)          # disjoint, contiguous seeds
    assert m0 == m1 == 125.0                                # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 608 / 0.125)       # all instances over the slowest time


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.replica_instances(0, 1, 608) == (0, 608)
