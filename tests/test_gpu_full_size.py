"""Full-size parity of the named workloads, at every step they define.

- 1e6 uniform points, 64x64 partitions, 1,000 steps of one 1-8-unit move per
  partition: the plain kinetic update, and the same steps with the trained locate
  proposal on.
- 16e6 mixture + lattice points, 256x256 partitions, 200 steps of 1-16 moves per
  partition.

After every step the GPU certificate (kdt_verify: every triangle counter-clockwise,
adjacency reciprocal, every edge locally Delaunay under SoS, 2n-2 live slots, the hull
winding once; together the definition of the unique triangulation) must find nothing.
At checkpoints the exported canonical list must equal the oracle's Bowyer-Watson
rebuild of the same positions, row for row.  The oracle runs in host threads while the
GPU steps (the move lists are drawn first, so every checkpoint's positions are known
before the first step)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same

pytestmark = pytest.mark.gpu

C2_STEPS = 1000
C2_CHECKS = (0, 1, 10, 100, 1000)
C3_STEPS = 200
C3_CHECKS = (0, 200)


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _draw(w, steps, checks):
    """All moves of `steps` steps, and the positions at each checkpoint."""
    snaps = {0: w.positions} if 0 in checks else {}
    moves = []
    for s in range(1, steps + 1):
        moves.append(w.next_moves())
        if s in checks:
            snaps[s] = w.positions
    return moves, snaps


@pytest.fixture(scope="module")
def c2_full():
    oracle.lib()
    w = W.c2()
    xy0 = w.positions
    moves, snaps = _draw(w, C2_STEPS, C2_CHECKS)
    pool = ThreadPoolExecutor(max(1, min(len(snaps), _cores())))
    fut = {s: pool.submit(oracle.delaunay, xy) for s, xy in snaps.items()}
    yield xy0, moves, snaps, fut
    pool.shutdown(wait=True)


def _run_checked(t, xy0, moves, snaps, checks):
    """Build, step through every move list with the certificate after every step, and
    keep the exported list at each checkpoint."""
    import torch
    t.build(torch.from_numpy(xy0).cuda())
    assert t.verify() == 0
    got = {0: t.export_triangles()} if 0 in checks else {}
    for s, mv in enumerate(moves, start=1):
        t.step(torch.from_numpy(mv).cuda())
        bad = t.verify()
        assert bad == 0, "step %d: %d certificate failures" % (s, bad)
        if s in checks:
            got[s] = t.export_triangles()
            assert np.array_equal(t.export_points(), snaps[s]), "positions at step %d" % s
    return got


def _compare(got, fut, what):
    for s in sorted(got):
        exp = fut[s].result()
        assert got[s].shape == exp.shape and np.array_equal(got[s], exp), \
            "%s: step %d differs from the oracle (%d vs %d rows)" % (what, s, got[s].shape[0], exp.shape[0])


def test_c2_full_size_all_steps(c2_full):
    from paper_2308_06484_gb300 import kdt
    xy0, moves, snaps, fut = c2_full
    t = kdt.Triangulation(kdt.default_config(grid=64, domain_bits=24))
    got = _run_checked(t, xy0, moves, snaps, C2_CHECKS)
    st = t.stats()
    assert st["moves"] == sum(m.shape[0] for m in moves)
    assert st["fallbacks"] == 0
    t.close()
    _compare(got, fut, "1e6 points")


def test_c2_full_size_with_trained_proposal(c2_full):
    """The same 1,000 steps with the locate proposal trained on its own (training-seed)
    traces: the triangulation stays bit-exact, whatever the network proposes."""
    from paper_2308_06484_gb300 import kdt, proposal
    xy0, moves, snaps, fut = c2_full
    x, y = proposal.collect_traces(proposal.default_training_sources())
    holder = kdt.Triangulation(kdt.default_config())
    tn = proposal.Trainer(holder, seed=0)
    tn.fit(x, y, epochs=4, batch=8192, seed=0)
    acc, _ = tn.evaluate(x, y)
    assert acc > 0.3
    t = kdt.Triangulation(kdt.default_config(grid=64, domain_bits=24))
    t.set_proposal(tn.params)
    got = _run_checked(t, xy0, moves, snaps, C2_CHECKS[1:])
    st = t.stats()
    assert st["proposal_moves"] > 0.5 * st["moves"]
    assert st["proposal_hits"] > 0.3 * st["proposal_moves"]
    t.close()
    holder.close()
    _compare(got, fut, "1e6 points, proposal on")


def test_c3_full_size_all_steps():
    """16e6 points over all 200 steps.  One oracle rebuild of 16e6 points takes a
    quarter of an hour, so the build and the last step are compared with the oracle
    tile by tile (assert_same_tiled: overlapping tiles triangulated by the oracle in
    parallel, their certified triangles, the exact empty-circle test for the rest, and
    Euler's count) -- the same row-for-row equality."""
    import torch
    from paper_2308_06484_gb300 import kdt
    from tests.gpu_helpers import assert_same_tiled
    oracle.lib()
    w = W.c3()
    xy0 = w.positions
    moves, snaps = _draw(w, C3_STEPS, C3_CHECKS)
    t = kdt.Triangulation(kdt.default_config(grid=256, domain_bits=24))
    got = _run_checked(t, xy0, moves, snaps, C3_CHECKS)
    st = t.stats()
    assert st["moves"] == sum(m.shape[0] for m in moves)
    assert st["moves"] > 100000 * C3_STEPS
    t.close()
    del t
    torch.cuda.empty_cache()
    for s in C3_CHECKS:
        assert_same_tiled(got[s], snaps[s], 24, tiles=16, overlap=1 / 16, what="16e6 points step %d" % s)
