"""Pins for the CPU oracle (no GPU).

Every check compares the oracle with something other than itself: hand-derived
fixtures, exact big-integer determinants of a different formula, the brute-force
empty-circle definition, an independent hull, Euler's formula, scipy's Qhull on
inputs proven free of ties, and order independence.
"""
import glob
import os

import numpy as np
import pytest

import oracle
from tests import _pins
from paper_2308_06484_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(path):
    pts, tris = [], []
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "P":
            pts.append((int(f[1]), int(f[2])))
        elif f[0] == "T":
            tris.append((int(f[1]), int(f[2]), int(f[3])))
    return np.array(pts, dtype=np.int32), sorted(tris)


def as_list(T):
    return [tuple(int(v) for v in r) for r in np.asarray(T)]


# ---------------------------------------------------------------- predicates

def _rand_pts(rng, m, lo, hi):
    return rng.integers(lo, hi, size=(m, 2), dtype=np.int64)


@pytest.mark.parametrize("span", [1 << 8, 1 << 20, 1 << 28])
def test_orient_matches_bigint_determinant(span):
    rng = np.random.default_rng(11)
    for _ in range(300):
        p = _rand_pts(rng, 3, 0, span).astype(np.int32)
        s = oracle.orient2d(p, 0, 1, 2)
        assert s == _pins.sign(_pins.orient_bigint(p[0], p[1], p[2]))


@pytest.mark.parametrize("span", [1 << 6, 1 << 20, 1 << 28])
def test_incircle_matches_lifted_4x4(span):
    rng = np.random.default_rng(12)
    for _ in range(400):
        p = _rand_pts(rng, 4, 0, span).astype(np.int32)
        s = oracle.incircle_raw(p, 0, 1, 2, 3)
        assert s == _pins.sign(_pins.det4_lifted(p))


def test_incircle_extreme_corners():
    # largest differences the API admits: coordinates at 0 and 2^28 - 1
    M = (1 << 28) - 1
    cases = [[(0, 0), (M, 0), (M, M), (0, M)],
             [(0, 0), (M, 0), (0, M), (M - 1, M - 1)],
             [(0, 0), (M, 1), (1, M), (M, M)],
             [(M, M), (0, M), (0, 0), (M, 0)]]
    for c in cases:
        p = np.array(c, dtype=np.int32)
        for perm in ([0, 1, 2, 3], [1, 2, 0, 3], [2, 1, 0, 3], [3, 1, 2, 0]):
            q = p[perm]
            assert oracle.incircle_raw(q, 0, 1, 2, 3) == _pins.sign(_pins.det4_lifted(q))


def test_incircle_sos_matches_perturbed_determinant():
    """Ties (cocircular quadruples of a lattice) against the evaluated perturbation."""
    rng = np.random.default_rng(13)
    grid = np.array([(x, y) for x in range(5) for y in range(5)], dtype=np.int32) * 37 + 5
    ties = 0
    for _ in range(3000):
        idx = rng.choice(len(grid), size=4, replace=False)
        xy = grid.copy()
        perm = rng.permutation(len(grid))
        xy = xy[perm]
        a, b, c, d = [int(np.nonzero(perm == i)[0][0]) for i in idx]
        if oracle.orient2d(xy, a, b, c) == 0:
            continue
        raw = oracle.incircle_raw(xy, a, b, c, d)
        ties += raw == 0
        assert oracle.incircle_sos(xy, a, b, c, d) == _pins.sos_incircle_bigint(xy, a, b, c, d)
    assert ties > 50


def test_incircle_sos_never_zero_for_distinct_points():
    rng = np.random.default_rng(14)
    grid = np.array([(x, y) for x in range(4) for y in range(4)], dtype=np.int32)
    for _ in range(2000):
        a, b, c, d = rng.choice(16, size=4, replace=False)
        if oracle.orient2d(grid, a, b, c) != 0:
            assert oracle.incircle_sos(grid, a, b, c, d) != 0


# ---------------------------------------------------------- triangulations

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))))
def test_golden_fixtures(path):
    if os.path.basename(path) == "README.txt":
        pytest.skip("readme")
    xy, expect = load_golden(path)
    assert as_list(oracle.delaunay(xy)) == expect
    assert oracle.check_dt(xy, np.array(expect)) == 0


def _small_sets():
    rng = np.random.default_rng(21)
    sets = []
    for n in (3, 4, 5, 7, 12, 20, 30):
        xy = np.unique(rng.integers(0, 1 << 10, size=(3 * n, 2)), axis=0)
        rng.shuffle(xy)
        sets.append(("uniform%d" % n, xy[:n]))
    for n in (9, 16, 25, 30):  # lattice: many cocircular quadruples
        xy = np.unique(rng.integers(0, 6, size=(6 * n, 2)), axis=0) * 3
        rng.shuffle(xy)
        sets.append(("lattice%d" % n, xy[:n]))
    # collinear-heavy: points on few lines, with hull segments holding many points
    line = np.array([(x, 0) for x in range(0, 40, 4)] + [(0, y) for y in range(4, 40, 4)]
                    + [(x, 40 - x) for x in range(4, 40, 4)])
    rng.shuffle(line)
    sets.append(("triangle_edges", line))
    pts = np.array([(x, 7) for x in range(12)] + [(5, 0), (6, 13), (3, 2), (9, 11)])
    rng.shuffle(pts)
    sets.append(("one_line_plus", pts))
    circ = np.array([(5, 0), (4, 3), (3, 4), (0, 5), (-3, 4), (-4, 3), (-5, 0), (-4, -3),
                     (-3, -4), (0, -5), (3, -4), (4, -3), (0, 0)]) + 10
    rng.shuffle(circ)
    sets.append(("circle12_center", circ))
    sets.append(("circle12", circ[np.any(circ != 10, axis=1)]))
    return sets


@pytest.mark.parametrize("name,xy", _small_sets(), ids=[s[0] for s in _small_sets()])
def test_oracle_equals_brute_force(name, xy):
    xy = np.asarray(xy, dtype=np.int32)
    got = as_list(oracle.delaunay(xy))
    assert got == _pins.brute_force_dt(xy)


@pytest.mark.parametrize("name,xy", _small_sets(), ids=[s[0] for s in _small_sets()])
def test_euler_and_hull(name, xy):
    xy = np.asarray(xy, dtype=np.int32)
    T = oracle.delaunay(xy)
    hull = _pins.hull_boundary(xy)
    assert _pins.boundary_edges_of(T) == hull
    h = len(hull)
    assert T.shape[0] == 2 * xy.shape[0] - 2 - h
    used = np.zeros(xy.shape[0], bool)
    used[T.ravel()] = True
    assert used.all()


def test_uniqueness_under_insertion_order():
    rng = np.random.default_rng(31)
    xy = np.unique(rng.integers(0, 20, size=(600, 2)), axis=0) * 5   # lattice ties
    rng.shuffle(xy)
    xy = xy[:300].astype(np.int32)
    ref = oracle.delaunay(xy, seed=1)
    for s in range(2, 12):
        assert np.array_equal(oracle.delaunay(xy, seed=s), ref)


def test_matches_scipy_in_general_position():
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(41)
    for n in (50, 500, 5000):
        xy = np.unique(rng.integers(0, 1 << 22, size=(n + 50, 2)), axis=0)
        rng.shuffle(xy)
        xy = xy[:n].astype(np.int32)
        T = oracle.delaunay(xy)
        # prove there is no tie: no interior edge of T has a cocircular opposite vertex
        edges = {}
        for t in T:
            for i in range(3):
                edges[(t[(i + 1) % 3], t[(i + 2) % 3])] = (tuple(t), t[i])
        for (a, b), (t, _) in edges.items():
            if (b, a) in edges:
                d = edges[(b, a)][1]
                assert oracle.incircle_raw(xy, t[0], t[1], t[2], d) != 0
        S = Delaunay(xy.astype(np.float64)).simplices
        canon = []
        for a, b, c in S:
            if oracle.orient2d(xy, a, b, c) < 0:
                b, c = c, b
            r = [int(a), int(b), int(c)]
            k = r.index(min(r))
            canon.append(tuple(r[k:] + r[:k]))
        assert sorted(canon) == as_list(T)


def test_workload_c1_initial_is_certified():
    w = W.c1()
    xy = w.positions
    T = oracle.delaunay(xy)
    assert oracle.check_dt(xy, T) == 0
    hull = _pins.hull_boundary(xy)
    assert T.shape[0] == 2 * xy.shape[0] - 2 - len(hull)


# ------------------------------------------------------------- error paths

def test_errors():
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[0, 0], [1, 1]]))
    assert e.value.code == -4
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[0, 0], [1, 1], [2, 2], [3, 3]]))
    assert e.value.code == -4
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[0, 0], [1, 0], [0, 1], [1, 0]]))
    assert e.value.code == -3
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[0, 0], [1, 0], [0, 1 << 28]]))
    assert e.value.code == -2


# ------------------------------------------------------------- certifier

def test_certifier_rejects_planted_mistakes():
    rng = np.random.default_rng(51)
    xy = np.unique(rng.integers(0, 1 << 12, size=(400, 2)), axis=0)
    rng.shuffle(xy)
    xy = xy[:300].astype(np.int32)
    T = oracle.delaunay(xy)
    assert oracle.check_dt(xy, T) == 0
    # 1: a clockwise triangle
    bad = T.copy(); bad[5, [1, 2]] = bad[5, [2, 1]]
    assert oracle.check_dt(xy, bad) != 0
    # a dropped triangle
    assert oracle.check_dt(xy, np.delete(T, 17, axis=0)) != 0
    # a duplicated triangle
    assert oracle.check_dt(xy, np.concatenate([T, T[:1]])) != 0
    # an interior edge flipped the wrong way (valid triangulation, not Delaunay)
    edges = {}
    for k, t in enumerate(T):
        for i in range(3):
            edges[(t[(i + 1) % 3], t[(i + 2) % 3])] = (k, t[i])
    flipped = None
    for (a, b), (k, c) in edges.items():
        if (b, a) in edges:
            k2, d = edges[(b, a)]
            # flip only if the new quad diagonal gives two ccw triangles
            if oracle.orient2d(xy, c, a, d) > 0 and oracle.orient2d(xy, d, b, c) > 0:
                flipped = T.copy()
                flipped[k] = (c, a, d)
                flipped[k2] = (d, b, c)
                break
    assert flipped is not None
    assert oracle.check_dt(xy, flipped) == 5
