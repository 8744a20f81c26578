"""The displacement rule of kdt_config.rebuild_displacement (the paper's abstract: when
points move far, rebuilding is cheaper; Section III: d, the N-th nearest-neighbour
distance, is the yardstick).  A step whose move goes farther than f * d_local of its
partition is done as a certified rebuild; the triangulation is the same as the
oracle's either way, and an invalid move still wins over the rule."""
import math

import numpy as np
import pytest

from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same, run_kinetic

pytestmark = pytest.mark.gpu


def _tri(w, f):
    from paper_2308_06484_gb300 import kdt
    t = kdt.Triangulation(kdt.default_config(grid=w.grid, domain_bits=w.bits, rebuild_displacement=f))
    t.build(w.positions)
    return t


def test_far_moves_take_the_rebuild():
    w = W.KineticWorkload(W.uniform_points(20000, 20, 9), 16, 20, (1, 4), (1000, 60000), seed=10, name="far")
    t = _tri(w, 1.0)
    run_kinetic(t, w, 6, every=1)
    st = t.stats()
    assert st["far_rebuilds"] > 0
    assert st["rebuilds"] >= st["far_rebuilds"]
    assert st["steps"] == 6
    assert t.verify() == 0


def test_short_moves_never_take_it():
    w = W.c1()
    t = _tri(w, 1.0)
    run_kinetic(t, w, 20, every=5)
    st = t.stats()
    assert st["far_rebuilds"] == 0 and st["deletes"] == st["moves"]


def test_threshold_is_strict_and_per_partition():
    """A move of squared length exactly f^2 * d_local^2 stays kinetic; one unit more
    takes the rebuild.  d_local^2 is the running per-partition minimum of the N-th
    nearest-neighbour squared distance, here read back through kdt_d_values."""
    from paper_2308_06484_gb300 import kdt
    xy = W.uniform_points(4000, 16, 21)
    t = kdt.Triangulation(kdt.default_config(grid=4, domain_bits=16, rebuild_displacement=1.0))
    t.build(xy)
    cm = np.empty(16, dtype=np.int64)
    t.d_values(1, cell_min2=cm)
    cur = xy.astype(np.int64).copy()
    cells = W.cell_of(cur, 4, 16)
    occupied = set(map(tuple, cur.tolist()))
    # d_local^2 = D is a squared distance between two points, so some (dx, dy) has
    # dx^2 + dy^2 = D exactly: a move by it sits on the bound; one unit more along x
    # goes beyond it
    done = []
    rng = np.random.default_rng(3)
    for beyond in (False, True):
        for p in rng.permutation(len(cur)):
            D = int(cm[cells[p]])
            dx = next(a for a in range(math.isqrt(D) + 1) if math.isqrt(D - a * a) ** 2 == D - a * a)
            dy = math.isqrt(D - dx * dx)
            q = (int(cur[p, 0]) + dx + (1 if beyond else 0), int(cur[p, 1]) + dy)
            if q[0] >= (1 << 16) or q[1] >= (1 << 16) or q in occupied or any(p == e[0] for e in done):
                continue
            L2 = (q[0] - int(cur[p, 0])) ** 2 + (q[1] - int(cur[p, 1])) ** 2
            done.append((int(p), q, L2 > D))
            break
    assert len(done) == 2 and not done[0][2] and done[1][2]
    for p, q, beyond in done:
        before = t.stats()["far_rebuilds"]
        t.step(np.array([[p, q[0], q[1]]], dtype=np.int32))
        occupied.discard(tuple(cur[p].tolist()))
        cur[p] = q
        occupied.add(q)
        assert t.stats()["far_rebuilds"] - before == (1 if beyond else 0)
        assert_same(t.export_triangles(), cur.astype(np.int32), "threshold move")
    assert t.verify() == 0


def test_invalid_move_wins_over_the_rule():
    from paper_2308_06484_gb300 import kdt
    w = W.KineticWorkload(W.uniform_points(20000, 20, 9), 16, 20, (1, 4), (1000, 60000), seed=10, name="far")
    t = _tri(w, 1.0)
    before = t.export_triangles()
    mv = w.next_moves()
    bad = np.concatenate([mv, np.array([[w.n + 5, 10, 10]], dtype=np.int32)])  # an id out of range
    with pytest.raises(kdt.KDTError) as e:
        t.step(bad)
    assert e.value.name == "KDT_ERR_ARG"
    assert t.stats()["far_rebuilds"] == 0
    assert np.array_equal(t.export_triangles(), before)
