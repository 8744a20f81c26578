"""Strip sharding with the seam exchange (paper_2308_06484_gb300/shard.py) on CPU ranks
(gloo), each rank's local triangulator being the oracle: after every step the union of
the ranks' shares equals the oracle's triangulation of all points, row for row, for two
and three ranks, with points crossing strips (hand-off), a halo that starts too thin
(the certificate widens it), and a clustered set."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleLocal:
    """A local triangulator for CPU tests: the oracle, rebuilt from scratch."""

    def build(self, xy):
        self.xy = np.array(xy, dtype=np.int32)

    def step(self, moves):
        m = np.asarray(moves, dtype=np.int64)
        self.xy[m[:, 0]] = m[:, 1:]

    def triangles(self):
        import oracle
        return oracle.delaunay(self.xy)


def _workload(kind):
    from paper_2308_06484_gb300 import workloads as W
    if kind == "uniform":
        return W.KineticWorkload(W.uniform_points(3000, 16, 81), 8, 16, (1, 2), (1, 400), seed=82, name="u")
    return W.KineticWorkload(W.mixture_lattice_points(3000, 16, 83, n_comp=4, sigma=4000.0, spacing=16), 8, 16,
                             (1, 2), (1, 300), seed=84, name="mix")


def _worker(rank, world, port, kind, halo, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2308_06484_gb300 import shard
        w = _workload(kind)
        sh = shard.StripShards(rank, world, w.grid, w.bits, halo, OracleLocal())
        xy = w.positions
        sh.start(np.arange(w.n), xy)
        results = []
        got = sh.gather_triangles()
        results.append(bool(np.array_equal(got, oracle.delaunay(xy))) if rank == 0 else True)
        crossed = 0
        for _ in range(steps):
            before = sh.owner_of(w.positions[:, 0])
            mv = w.next_moves()
            crossed += int(np.count_nonzero(sh.owner_of(mv[:, 1]) != before[mv[:, 0]]))
            sh.step(mv)
            got = sh.gather_triangles()
            if rank == 0:
                results.append(bool(np.array_equal(got, oracle.delaunay(w.positions))))
        q.put((rank, results, crossed, sh.widenings, sh.rebuilds, sh.halo))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(world, kind, halo, steps=6):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, halo, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world,kind", [(2, "uniform"), (3, "mixture")])
def test_sharded_union_equals_the_whole_triangulation(world, kind):
    res = _run(world, kind, halo=4096)
    rank0 = res[0]
    assert all(rank0[1]), rank0[1]          # build and every step, row for row
    assert sum(r[2] for r in res) > 0       # points were handed to another strip
    assert all(r[4] >= 1 for r in res)


def test_too_thin_halo_is_widened_by_the_certificate():
    res = _run(2, "uniform", halo=1, steps=3)
    assert all(res[0][1])
    assert res[0][3] > 0 and res[0][5] > 1  # widened at least once
