"""The multi-rank bench aggregation (replicas: sum of updates, max of times) on two
gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    u, t, e = bench.aggregate(1000.0 * (rank + 1), 2.0 + rank, 3.0 - rank)
    q.put((rank, u, t, e))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, u, t, e in res:
        assert u == 3000.0      # updates summed over ranks
        assert t == 3.0         # timed region: max over ranks
        assert e == 3.0


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(10.0, 2.0, 3.0) == (10.0, 2.0, 3.0)
