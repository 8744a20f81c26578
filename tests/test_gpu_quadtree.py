"""Quad-tree partitions (kdt_config.quadtree, Section III "Data structure") on the GPU:
the leaves equal the reference in oracle/quadtree.py (their number, and every point's
leaf through the per-leaf minima of kdt_d_values, before and after moves), and steps
scheduled on them give the oracle's triangulation after every step."""
import numpy as np
import pytest

from oracle import dcalc as D
from oracle import quadtree as Q
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same, run_kinetic

pytestmark = pytest.mark.gpu


def _tri(**kw):
    from paper_2308_06484_gb300 import kdt
    kw.setdefault("quadtree", 1)
    return kdt.Triangulation(kdt.default_config(**kw))


def _leaf_minima(t, xy, sq, lay, N=2):
    cmin = np.empty(len(sq), dtype=np.int64)
    t.d_values(N, None, cmin)
    exp = np.full(len(sq), D.NONE, dtype=np.int64)
    np.minimum.at(exp, Q.block_of(xy, sq, lay), D.nth_nn_dist2(xy, N))
    assert np.array_equal(cmin, exp)


@pytest.mark.parametrize("T", [16, 64, 256])
def test_leaves_match_reference(T):
    xy = W.mixture_lattice_points(30000, 24, 21)
    t = _tri(domain_bits=24, points_per_partition=T)
    t.build(xy)
    sq, lay = Q.leaves(xy, T)
    assert t.num_cells() == len(sq)
    _leaf_minima(t, xy, sq, lay)


def test_blocks_follow_moves():
    import torch
    w = W.KineticWorkload(W.mixture_lattice_points(20000, 24, 23), 32, 24, (1, 4), (1, 8), seed=24,
                          name="mix-qt")
    t = _tri(domain_bits=24, points_per_partition=64)
    t.build(w.positions)
    sq, lay = Q.leaves(w.positions, 64)  # the tree of the build positions stays
    for s in range(4):
        t.step(torch.from_numpy(w.next_moves()).cuda())
        assert_same(t.export_triangles(), w.positions, "quadtree step %d" % s)
    _leaf_minima(t, w.positions, sq, lay)
    assert t.num_cells() == len(sq)


@pytest.mark.parametrize("make", [lambda: W.c1(), lambda: W.c2(n=50000, grid=32, seed=25)])
def test_kinetic_parity(make):
    w = make()
    t = _tri(domain_bits=w.bits, points_per_partition=64)
    t.build(w.positions)
    t.reset_stats()
    run_kinetic(t, w, 10, every=1)
    st = t.stats()
    assert st["fallbacks"] == 0
    assert t.verify() == 0


def test_batch_rejected():
    from paper_2308_06484_gb300 import kdt
    t = _tri(domain_bits=20)
    with pytest.raises(kdt.KDTError):
        t.build_batch([W.uniform_points(100, 20, 1), W.uniform_points(100, 20, 2)])


def test_redivided_at_every_step():
    """kdt_config.quadtree = 2: the division is made again on the GPU at the start of
    every step (Fig. 4), inside the build's square; after each step the leaves in use
    are the reference's division of the positions the step started from, every point's
    leaf follows through the per-leaf minima, and the triangulation equals the oracle's."""
    import torch
    w = W.KineticWorkload(W.mixture_lattice_points(20000, 20, 27), 16, 20, (1, 4), (500, 40000), seed=28,
                          name="qt-every-step")
    t = _tri(domain_bits=20, points_per_partition=48, quadtree=2)
    t.build(w.positions)
    sq0, lay = Q.leaves(w.positions, 48)
    assert t.num_cells() == len(sq0)
    counts = set()
    for s in range(6):
        before = w.positions
        t.step(torch.from_numpy(w.next_moves()).cuda())
        assert_same(t.export_triangles(), w.positions, "re-divided quadtree step %d" % s)
        sq, _ = Q.leaves(before, 48, lay=lay)
        assert t.num_cells() == len(sq), (s, t.num_cells(), len(sq))
        _leaf_minima(t, w.positions, sq, lay)
        counts.add(len(sq))
    assert len(counts) > 1  # the division changed over the steps
    assert t.verify() == 0
