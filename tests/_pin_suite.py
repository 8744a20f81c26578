"""Run the oracle's pins against one oracle build; used to show each pin bites.

``python -m tests._pin_suite <liboracle.so>`` exits 0 when every pin holds and 1
when any fails (a crash of a broken build also gives a non-zero status).
"""
import glob
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests import _pins  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _canon_list(T):
    return [tuple(int(v) for v in r) for r in np.asarray(T)]


def _load_golden(path):
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


def pin_golden(o):
    for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))):
        if p.endswith("README.txt"):
            continue
        xy, expect = _load_golden(p)
        if _canon_list(o.delaunay(xy)) != expect:
            return False
    return True


def pin_predicates(o):
    rng = np.random.default_rng(7)
    for _ in range(200):
        p = rng.integers(0, 1 << 20, size=(4, 2)).astype(np.int32)
        if o.orient2d(p, 0, 1, 2) != _pins.sign(_pins.orient_bigint(p[0], p[1], p[2])):
            return False
        if o.incircle_raw(p, 0, 1, 2, 3) != _pins.sign(_pins.det4_lifted(p)):
            return False
    grid = np.array([(x, y) for x in range(4) for y in range(4)], dtype=np.int32) * 3
    for _ in range(400):
        a, b, c, d = [int(v) for v in rng.choice(16, size=4, replace=False)]
        if o.orient2d(grid, a, b, c) == 0:
            continue
        if o.incircle_sos(grid, a, b, c, d) != _pins.sos_incircle_bigint(grid, a, b, c, d):
            return False
    return True


def _sets():
    rng = np.random.default_rng(5)
    out = []
    for n in (6, 15, 25):
        xy = np.unique(rng.integers(0, 1 << 10, size=(3 * n, 2)), axis=0)
        rng.shuffle(xy)
        out.append(xy[:n].astype(np.int32))
    xy = np.unique(rng.integers(0, 5, size=(80, 2)), axis=0) * 4
    rng.shuffle(xy)
    out.append(xy[:20].astype(np.int32))
    out.append(np.array([(x, 0) for x in range(8)] + [(3, 5), (6, 2), (1, 9)], dtype=np.int32))
    return out


def pin_brute_force(o):
    for xy in _sets():
        if _canon_list(o.delaunay(xy)) != _pins.brute_force_dt(xy):
            return False
    return True


def pin_euler_hull(o):
    for xy in _sets():
        T = o.delaunay(xy)
        hull = _pins.hull_boundary(xy)
        if _pins.boundary_edges_of(T) != hull:
            return False
        if T.shape[0] != 2 * xy.shape[0] - 2 - len(hull):
            return False
    return True


def pin_order_independence(o):
    rng = np.random.default_rng(9)
    xy = (np.unique(rng.integers(0, 12, size=(300, 2)), axis=0) * 3).astype(np.int32)
    rng.shuffle(xy)
    ref = o.delaunay(xy, seed=1)
    return all(np.array_equal(o.delaunay(xy, seed=s), ref) for s in range(2, 7))


def pin_scipy(o):
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(3)
    xy = np.unique(rng.integers(0, 1 << 22, size=(2100, 2)), axis=0)
    rng.shuffle(xy)
    xy = xy[:2000].astype(np.int32)
    S = Delaunay(xy.astype(np.float64)).simplices
    canon = []
    for a, b, c in S:
        if _pins.orient_bigint(xy[a], xy[b], xy[c]) < 0:
            b, c = c, b
        r = [int(a), int(b), int(c)]
        k = r.index(min(r))
        canon.append(tuple(r[k:] + r[:k]))
    return sorted(canon) == _canon_list(o.delaunay(xy))


PINS = [pin_golden, pin_predicates, pin_brute_force, pin_euler_hull,
        pin_order_independence, pin_scipy]


def run_all(o):
    failed = []
    for pin in PINS:
        try:
            ok = pin(o)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    return failed


if __name__ == "__main__":
    o = oracle.Oracle(sys.argv[1] if len(sys.argv) > 1 else None)
    failed = run_all(o)
    print("failed pins:", failed)
    sys.exit(1 if failed else 0)
