"""Kinetic steps (delete + insert per moved point, Fig. 4) against the oracle after
every step, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same, run_kinetic

pytestmark = pytest.mark.gpu


def _tri(**kw):
    from paper_2308_06484_gb300 import kdt
    return kdt.Triangulation(kdt.default_config(**kw))


def _setup(w, **kw):
    t = _tri(grid=w.grid, domain_bits=w.bits, **kw)
    t.build(w.positions)
    assert_same(t.export_triangles(), w.positions, "initial")
    t.reset_stats()
    return t


def test_c1_all_100_steps():
    w = W.c1()
    t = _setup(w)
    run_kinetic(t, w, 100, every=1)
    st = t.stats()
    assert st["fallbacks"] == 0
    assert st["deletes"] == st["inserts"] == st["moves"] == 1600
    assert t.verify() == 0


def test_c2_shaped_small():
    w = W.c2(n=100000, grid=64)
    t = _setup(w)
    run_kinetic(t, w, 10, every=1)
    assert t.stats()["fallbacks"] == 0


def test_many_moves_per_cell():
    w = W.KineticWorkload(W.uniform_points(60000, 24, 5), 32, 24, (1, 16), (1, 8), seed=6, name="multi")
    t = _setup(w)
    run_kinetic(t, w, 6, every=1)
    assert t.stats()["fallbacks"] == 0


def test_mixture_lattice_moves():
    w = W.KineticWorkload(W.mixture_lattice_points(100000, 24, 7), 64, 24, (1, 16), (1, 8), seed=8,
                          name="c3-shaped")
    t = _setup(w)
    run_kinetic(t, w, 5, every=1)
    st = t.stats()
    assert st["fallbacks"] == 0
    assert st["sos_ties"] > 0


def test_large_moves_cross_partitions():
    w = W.KineticWorkload(W.uniform_points(20000, 20, 9), 16, 20, (1, 4), (1000, 60000), seed=10,
                          name="far")
    t = _setup(w)
    run_kinetic(t, w, 8, every=1)
    assert t.stats()["fallbacks"] == 0


def test_hull_moves_and_outside():
    """Move hull points outwards and inwards, and points to outside the hull."""
    rng = np.random.default_rng(12)
    xy = W.uniform_points(3000, 16, 12).astype(np.int64)
    xy = (xy // 4 + (1 << 13)).astype(np.int32)  # points in the middle of the domain
    t = _tri(grid=4, domain_bits=16)
    t.build(xy)
    cur = xy.copy()
    occupied = set(map(tuple, cur.tolist()))
    for s in range(10):
        hullv = np.unique(np.array(oracle.delaunay(cur)).ravel())
        ids = rng.choice(len(cur), size=40, replace=False)
        mv = []
        for i in ids:
            for _ in range(50):
                tgt = (int(rng.integers(0, 1 << 16)), int(rng.integers(0, 1 << 16)))
                if tgt not in occupied:
                    break
            occupied.discard(tuple(cur[i]))
            occupied.add(tgt)
            mv.append((i, tgt[0], tgt[1]))
            cur[i] = tgt
        t.step(np.array(mv, dtype=np.int32))
        assert_same(t.export_triangles(), cur, "hull step %d" % s)
    assert t.verify() == 0


def test_points_landing_on_edges_and_lines():
    """Targets exactly on existing edges and on hull segments (2->4 splits)."""
    g = np.array([(x, y) for x in range(20) for y in range(20)], dtype=np.int32) * 8
    rng = np.random.default_rng(13)
    t = _tri(grid=4, domain_bits=16)
    cur = g.copy()
    t.build(cur)
    occupied = set(map(tuple, cur.tolist()))
    for s in range(10):
        ids = rng.choice(len(cur), size=12, replace=False)
        mv = []
        for i in ids:
            for _ in range(100):
                # midpoints of lattice edges lie on existing edges or cocircular spots
                tgt = (int(rng.integers(0, 40)) * 4, int(rng.integers(0, 40)) * 4)
                if tgt not in occupied:
                    break
            occupied.discard(tuple(cur[i]))
            occupied.add(tgt)
            mv.append((i, tgt[0], tgt[1]))
            cur[i] = tgt
        t.step(np.array(mv, dtype=np.int32))
        assert_same(t.export_triangles(), cur, "edge step %d" % s)
    st = t.stats()
    assert st["edge_splits"] > 0
    assert t.verify() == 0


def test_swap_and_chain_targets():
    """Targets on positions vacated in the same step (deferred insertion)."""
    xy = W.uniform_points(500, 12, 14)
    t = _tri(grid=4, domain_bits=12)
    t.build(xy)
    cur = xy.copy()
    # a swap (two points exchange places) and a chain a->b->c->free
    mv = np.array([(0, cur[1, 0], cur[1, 1]), (1, cur[0, 0], cur[0, 1]),
                   (2, cur[3, 0], cur[3, 1]), (3, cur[4, 0], cur[4, 1]), (4, 4095, 4095)], dtype=np.int32)
    assert (4095, 4095) not in set(map(tuple, cur.tolist()))
    for i, x, y in mv:
        cur[i] = (x, y)
    t.step(mv)
    assert_same(t.export_triangles(), cur, "swap/chain")
    assert t.verify() == 0


def test_step_errors_leave_state_unchanged():
    from paper_2308_06484_gb300 import kdt
    w = W.c1()
    t = _setup(w)
    before = t.export_triangles().copy()
    cur = w.positions
    bad_cases = {
        "KDT_ERR_ARG": [(1000, 5, 5)],
        "KDT_ERR_RANGE": [(3, 70000, 5)],
        "KDT_ERR_DUPLICATE": [(3, 5, 5), (3, 6, 6)],
    }
    for name, mv in bad_cases.items():
        with pytest.raises(kdt.KDTError) as e:
            t.step(np.array(mv, dtype=np.int32))
        assert e.value.name == name
        assert np.array_equal(t.export_triangles(), before)
    # target on a point that does not move: a duplicate found while the step runs
    mv = np.array([(3, cur[10, 0], cur[10, 1])], dtype=np.int32)
    with pytest.raises(kdt.KDTError) as e:
        t.step(mv)
    assert e.value.name == "KDT_ERR_DUPLICATE"
    assert np.array_equal(t.export_triangles(), before)
    assert np.array_equal(t.export_points(), cur)
    # two moves onto the same free position
    mv = np.array([(3, 12345, 54321), (4, 12345, 54321)], dtype=np.int32)
    with pytest.raises(kdt.KDTError) as e:
        t.step(mv)
    assert e.value.name == "KDT_ERR_DUPLICATE"
    assert np.array_equal(t.export_triangles(), before)
    # an empty step is a no-op
    t.step(np.zeros((0, 3), dtype=np.int32))
    assert np.array_equal(t.export_triangles(), before)
    assert t.verify() == 0


def test_tiny_sets_and_degenerate_steps():
    """n = 3..6: every step touches the whole triangulation; collinear end states fail
    with KDT_ERR_DEGENERATE and leave the state unchanged."""
    from paper_2308_06484_gb300 import kdt
    rng = np.random.default_rng(15)
    for n in (3, 4, 5, 6):
        xy = W.uniform_points(n, 8, 100 + n)
        t = _tri(grid=2, domain_bits=8)
        t.build(xy)
        cur = xy.copy()
        for s in range(20):
            i = int(rng.integers(0, n))
            occ = set(map(tuple, cur.tolist()))
            while True:
                tgt = (int(rng.integers(0, 256)), int(rng.integers(0, 256)))
                if tgt not in occ:
                    break
            new = cur.copy()
            new[i] = tgt
            try:
                oracle.delaunay(new)
                ok = True
            except oracle.OracleError:
                ok = False
            if ok:
                t.step(np.array([(i, tgt[0], tgt[1])], dtype=np.int32))
                cur = new
            else:
                with pytest.raises(kdt.KDTError):
                    t.step(np.array([(i, tgt[0], tgt[1])], dtype=np.int32))
            assert_same(t.export_triangles(), cur, "tiny n=%d step %d" % (n, s))
    # make 4 points collinear by a move
    xy = np.array([(0, 0), (10, 0), (20, 0), (5, 9)], dtype=np.int32)
    t = _tri(grid=2, domain_bits=8)
    t.build(xy)
    with pytest.raises(kdt.KDTError) as e:
        t.step(np.array([(3, 30, 0)], dtype=np.int32))
    assert e.value.name == "KDT_ERR_DEGENERATE"
    assert_same(t.export_triangles(), xy, "collinear rejected")


def test_fallback_rebuild_and_retry_cap():
    """A forced retry cap of 1 either completes normally or falls back to the
    certified rebuild: the result is the same triangulation."""
    w = W.c2(n=50000, grid=64)
    t = _setup(w, retry_cap=1)
    run_kinetic(t, w, 5, every=1)
    w2 = W.c2(n=50000, grid=64)
    t2 = _setup(w2, rebuild_ratio=0.0001)  # every step is done as a full rebuild
    run_kinetic(t2, w2, 3, every=1)
    assert t2.stats()["rebuilds"] == 3  # one full rebuild per step


@pytest.mark.parametrize("make", [lambda: W.c1(), lambda: W.c2(n=30000, grid=16, seed=44),
                                  lambda: W.KineticWorkload(W.mixture_lattice_points(30000, 24, 45), 16, 24,
                                                            (1, 16), (1, 8), seed=46, name="mix")])
@pytest.mark.parametrize("variant", [1, 2])
def test_variant_in_place_moves(make, variant):
    """kdt_config.variant = 1 (move in place when the star stays Delaunay, else delete +
    insert) and 2 (move in place when the star stays counter-clockwise, the star's
    failing edges flipped by the step's repair) give the oracle's triangulation after
    every step."""
    w = make()
    t = _setup(w, variant=variant)
    run_kinetic(t, w, 8, every=1)
    st = t.stats()
    assert st["fallbacks"] == 0
    assert st["deletes"] < st["moves"]  # some moves were done in place
    assert t.verify() == 0


def _row_points(seed):
    """A straight row of 1000 points (spacing 64) with a few points beside it at heights
    of 600-2500 (each with a hundred or more row points in its star: degrees above the
    64 a shared-memory star holds), some of them with a companion a few units away (so
    that a short move can turn a triangle of the star over), and background points far
    from the row."""
    rng = np.random.default_rng(seed)
    y0 = 1 << 21
    row = np.stack([30000 + 64 * np.arange(1000), np.full(1000, y0)], 1)
    xs = 30000 + np.linspace(3000, 60000, 8).astype(np.int64) + 29
    hs = np.array([650, 900, 1400, 2500, -700, -1000, -1600, -2300])
    side = np.stack([xs, y0 + hs], 1)
    comp = side[[0, 2, 5, 7]] + np.array([[5, 3], [-4, 6], [6, -2], [3, 5]])
    bg = rng.integers(0, 1 << 22, size=(6000, 2))
    bg = bg[np.abs(bg[:, 1] - y0) > 60000][:2000]
    xy = np.concatenate([row, side, comp, bg]).astype(np.int32)
    assert np.unique(xy, axis=0).shape[0] == xy.shape[0]
    return xy, np.arange(1000, 1012)


def test_high_degree_points_move():
    """Points of degree above 64 (star in the warp's global scratch) moved by 1-8 units
    every step, beside and across their companions' edges: moved in place (with flips
    where the star stays valid but not Delaunay) or deleted (incremental ear clipping
    over a link of ~100 collinear row points) and inserted; the oracle's triangulation
    after every step."""
    import torch
    from paper_2308_06484_gb300 import kdt
    xy, movers = _row_points(61)
    t = kdt.Triangulation(kdt.default_config(grid=16, domain_bits=22))
    t.build(xy)
    assert_same(t.export_triangles(), xy, "initial")
    t.reset_stats()
    rng = np.random.default_rng(62)
    occ = set(map(tuple, xy.tolist()))
    dirs = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    for s in range(12):
        mv = []
        ids = list(movers) + list(rng.choice(np.arange(1012, xy.shape[0]), 20, replace=False))
        for p in ids:
            for _ in range(16):
                dx, dy = dirs[int(rng.integers(0, 4))]
                k = int(rng.integers(1, 9))
                q = (int(xy[p, 0]) + dx * k, int(xy[p, 1]) + dy * k)
                if 0 <= q[0] < 1 << 22 and 0 <= q[1] < 1 << 22 and q not in occ:
                    occ.discard(tuple(xy[p].tolist()))
                    occ.add(q)
                    xy[p] = q
                    mv.append((p, q[0], q[1]))
                    break
        t.step(torch.from_numpy(np.array(mv, dtype=np.int32)).cuda())
        assert_same(t.export_triangles(), xy, "row step %d" % s)
    st = t.stats()
    assert st["fallbacks"] == 0
    assert st["big_moves"] > 0
    assert t.verify() == 0
