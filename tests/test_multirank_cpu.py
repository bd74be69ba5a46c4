"""The benchmark's N > 1 path on CPU: two gloo ranks, each timing its own
replica; the job time is the slowest rank's and the work is summed (the
bench's whole-job throughput), and a rank that raises is reported instead of
hanging the other."""
from __future__ import annotations

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 20.0 - rank]          # rank 1 slower on the first
        units = [1000.0 * (rank + 1), 7.0]
        t, u = bench.reduce_over_ranks(times, units)
        q.put((rank, t, u))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in res:
        assert t == [11.0, 20.0]                  # max over ranks
        assert u == [3000.0, 14.0]                # sum over ranks


def _failing_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import datetime
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((rank, "raised"))
        raise SystemExit(3)                       # leaves between steps, no collective in flight
    try:
        bench.reduce_over_ranks([1.0], [1.0])
        q.put((rank, "completed"))
    except Exception as e:                        # the peer is gone: the collective errors out
        q.put((rank, type(e).__name__))


def test_peer_failure_surfaces_as_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "raised"
    assert res[0] != "completed"
    assert procs[1].exitcode == 3
