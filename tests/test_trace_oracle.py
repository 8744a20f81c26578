"""Pins for the CPU reference of the proposal's training rows (no GPU).

Against the hand-derived fixture tests/golden/diamond_move.trace, and on random
point sets against facts computed another way: Euler's relation for the cavity
size, the area of the link polygon for the hole triangles, an angular sort in
float64 for the wedge start, and a winding-number test for "beyond".
"""
import math
import os
from fractions import Fraction

import numpy as np

import oracle
from oracle import trace_ref as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "diamond_move.trace")


def _frac(s):
    return float(Fraction(s))


def load_trace_golden(path=GOLDEN):
    pts, moves = [], []
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "P":
            pts.append((int(f[1]), int(f[2])))
        elif f[0] == "M":
            p, qx, qy, slot, conflict = (int(x) for x in f[1:6])
            feats = np.array([_frac(x) for x in f[6:]], dtype=np.float64)
            assert feats.shape == (32,)
            moves.append((p, (qx, qy), slot, conflict, feats))
    return np.array(pts, dtype=np.int32), moves


def test_golden_diamond():
    xy, moves = load_trace_golden()
    assert len(moves) == 4
    for p, q, slot, conflict, feats in moves:
        f, s, c, _ = T.row(xy, p, q)
        assert (s, c) == (slot, conflict), (q, s, c)
        assert np.allclose(f, feats, rtol=2e-7, atol=1e-7), (q, f, feats)


def _area2(pts):
    a = 0
    for i in range(len(pts)):
        x0, y0 = pts[i]
        x1, y1 = pts[(i + 1) % len(pts)]
        a += int(x0) * int(y1) - int(x1) * int(y0)
    return a


def _winding_inside(poly, q):
    """Strictly inside a simple ccw polygon, by the angle sum (float64)."""
    tot = 0.0
    for i in range(len(poly)):
        ax, ay = poly[i][0] - q[0], poly[i][1] - q[1]
        bx, by = poly[(i + 1) % len(poly)][0] - q[0], poly[(i + 1) % len(poly)][1] - q[1]
        tot += math.atan2(ax * by - ay * bx, ax * bx + ay * by)
    return abs(tot) > math.pi


def test_invariants_random_sets():
    rng = np.random.default_rng(21)
    rows = 0
    slots = set()
    for trial in range(40):
        n = 40
        xy = rng.integers(0, 1 << 10, size=(n, 2)).astype(np.int32)
        if np.unique(xy, axis=0).shape[0] != n:
            continue
        T0 = oracle.delaunay(xy)
        for p in rng.choice(n, 6, replace=False):
            link = T.link_ccw(T0, int(p))
            if link is None:
                continue
            d = [(1, 0), (-1, 0), (0, 1), (0, -1)][rng.integers(0, 4)]
            dist = int(rng.integers(1, 120))
            q = (int(xy[p][0]) + d[0] * dist, int(xy[p][1]) + d[1] * dist)
            if not (0 <= q[0] < 1 << 10 and 0 <= q[1] < 1 << 10):
                continue
            if any((int(a) == q[0] and int(b) == q[1]) for a, b in xy):
                continue
            res = T.row(xy, int(p), q)
            f, slot, conflict, info = res
            k = len(link)
            rows += 1
            slots.add(slot)
            # hole triangles: k - 2 of them, tiling the link polygon
            hole = info["hole"]
            assert len(hole) == k - 2
            assert sum(_area2([xy[v] for v in t]) for _, t in hole) == _area2([xy[v] for v in link])
            # wedge start: the angular position of d among the link directions (float64)
            ang = [math.atan2(int(xy[v][1]) - int(xy[p][1]), int(xy[v][0]) - int(xy[p][0])) for v in link]
            ad = math.atan2(d[1], d[0])
            j0 = info["j0"]
            rel = lambda a: (a - ang[j0]) % (2 * math.pi)
            assert rel(ad) < rel(ang[(j0 + 1) % k]) or k == 1
            # beyond iff q is outside the closed link polygon
            inside = _winding_inside([xy[v] for v in link], q)
            on_boundary = any(T._orient(xy[link[i]], xy[link[(i + 1) % k]], q) == 0 and
                              min(xy[link[i]][0], xy[link[(i + 1) % k]][0]) <= q[0] <=
                              max(xy[link[i]][0], xy[link[(i + 1) % k]][0]) and
                              min(xy[link[i]][1], xy[link[(i + 1) % k]][1]) <= q[1] <=
                              max(xy[link[i]][1], xy[link[(i + 1) % k]][1]) for i in range(k))
            if k - 2 <= 16:
                assert (slot < 16) == (inside or on_boundary)
            # cavity size: Euler on the star of q in DT(P') when q is inside the hull
            T2 = info["T2"]
            deg_q = int(np.sum(np.any(T2 == p, axis=1)))
            l2 = T.link_ccw(T2, int(p))
            if l2 is not None:
                assert conflict == deg_q - 2
            assert f.dtype == np.float32 and f[1] == np.float32(k) / 16
    assert rows > 100
    assert len(slots) >= 4
