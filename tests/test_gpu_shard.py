"""The strip sharding (paper_2308_06484_gb300/shard.py) with the CUDA library as each
rank's local triangulator: two ranks (processes) on the one GPU of this run, exchanging
through gloo on the host (their kernels never wait on one another).  After the build and
every step the union of the ranks' shares equals the oracle's triangulation of all
points, row for row."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, steps, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2308_06484_gb300 import shard, workloads as W
        torch.cuda.set_device(0)
        w = W.KineticWorkload(W.uniform_points(20000, 20, 91), 8, 20, (1, 4), (1, 2000), seed=92, name="shard")
        local = shard.KdtLocal(20, device=0, grid=8)
        sh = shard.StripShards(rank, world, w.grid, w.bits, 8192, local)
        sh.start(np.arange(w.n), w.positions)
        ok = [bool(np.array_equal(sh.gather_triangles(), oracle.delaunay(w.positions)))] if rank == 0 else []
        kinetic_steps = 0
        for _ in range(steps):
            before = sh.rebuilds
            sh.step(w.next_moves())
            kinetic_steps += sh.rebuilds == before
            got = sh.gather_triangles()
            if rank == 0:
                ok.append(bool(np.array_equal(got, oracle.delaunay(w.positions))))
        local.close()
        q.put((rank, ok, kinetic_steps, sh.widenings))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_on_the_library():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 5, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(res[0][1]) and len(res[0][1]) == 6, res[0][1]
