"""Shared helpers of the GPU parity tests (compare the CUDA path with the oracle)."""
import numpy as np

import oracle


def assert_same(got, xy, what=""):
    exp = oracle.delaunay(xy)
    if got.shape != exp.shape or not np.array_equal(got, exp):
        g = set(map(tuple, got.tolist()))
        e = set(map(tuple, exp.tolist()))
        raise AssertionError("%s: GPU %d rows vs oracle %d rows; %d missing, %d extra; first missing %s"
                             % (what, got.shape[0], exp.shape[0], len(e - g), len(g - e),
                                sorted(e - g)[:3]))


def run_kinetic(tri, w, steps, every=1, check_points=True):
    """Apply `steps` generated steps; compare with the oracle every `every` steps."""
    import torch
    for s in range(steps):
        mv = w.next_moves()
        tri.step(torch.from_numpy(mv).cuda())
        if (s + 1) % every == 0 or s == steps - 1:
            if check_points:
                assert np.array_equal(tri.export_points(), w.positions)
            assert_same(tri.export_triangles(), w.positions, "%s step %d" % (w.name, s + 1))


def hull_count(xy):
    """Points on the convex hull boundary of distinct points, collinear ones included
    (monotone chain, exact integers).  Points strictly inside the polygon of the extreme
    points in 16 directions cannot be on the boundary and are dropped first."""
    pts = np.asarray(xy, dtype=np.int64).reshape(-1, 2)
    if pts.shape[0] < 3:
        return pts.shape[0]
    if pts.shape[0] > 64:
        ang = np.arange(16) * (2 * np.pi / 16)
        dirs = np.stack([np.round(1024 * np.cos(ang)), np.round(1024 * np.sin(ang))], axis=1).astype(np.int64)
        ext = np.array([np.argmax(pts[:, 0] * dx + pts[:, 1] * dy) for dx, dy in dirs])
        poly = [pts[i] for k, i in enumerate(ext) if k == 0 or i != ext[k - 1]]
        if len(poly) >= 3 and not np.array_equal(poly[0], poly[-1]):
            inside = np.ones(pts.shape[0], dtype=bool)
            for k in range(len(poly)):
                a, b = poly[k], poly[(k + 1) % len(poly)]
                inside &= (b[0] - a[0]) * (pts[:, 1] - a[1]) - (b[1] - a[1]) * (pts[:, 0] - a[0]) > 0
            pts = pts[~inside]

    def chain(P):
        h = []
        for p in P.tolist():
            while len(h) >= 2 and (h[-1][0] - h[-2][0]) * (p[1] - h[-2][1]) - (h[-1][1] - h[-2][1]) * (p[0] - h[-2][0]) < 0:
                h.pop()
            h.append((p[0], p[1]))
        return h
    pts = pts[np.lexsort((pts[:, 1], pts[:, 0]))]
    lower, upper = chain(pts), chain(pts[::-1])
    return len(set(lower) | set(upper))


def assert_same_tiled(got, xy, bits, tiles=8, overlap=0.5, threads=None, what=""):
    """`got` (canonical list of a large triangulation) equals the oracle's triangulation
    of xy, checked without one oracle call over all points: the domain is cut into
    tiles x tiles squares, each widened by `overlap` x its side on every side, and the
    oracle triangulates each widened tile's points (in parallel threads).  A tile's
    triangle whose circumcircle, inside the bounding box of all points, lies within the
    widened tile (with a margin) has no other point of the whole set in its circle, so it
    is a triangle of the whole set's triangulation.  Every such triangle must be in
    `got`; every row of `got` must be such a triangle of some tile, or pass the exact
    empty-circle test against every point near its circle; and `got` must have
    2n - 2 - h rows (h from an independent hull).  Together: `got` is the oracle's
    triangulation, row for row."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    from paper_2308_06484_gb300.shard import _x_extent_circle
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    L = 1 << bits
    side = L // tiles
    pad = int(side * overlap)
    bbox = tuple(float(v) for v in (xy[:, 0].min(), xy[:, 1].min(), xy[:, 0].max(), xy[:, 1].max()))
    x64 = xy.astype(np.int64)

    def one(k):
        i, j = divmod(k, tiles)
        x0, x1 = i * side - pad, (i + 1) * side + pad
        y0, y1 = j * side - pad, (j + 1) * side + pad
        sel = np.nonzero((x64[:, 0] >= x0) & (x64[:, 0] < x1) & (x64[:, 1] >= y0) & (x64[:, 1] < y1))[0]
        if sel.shape[0] < 3:
            return np.zeros((0, 3), np.int64)
        t = sel[oracle.delaunay(xy[sel])]
        P = x64[t].astype(np.float64)
        lo, hi, empty = _x_extent_circle(P, bbox)
        # the same test along y (swap the axes)
        Py = P[:, :, ::-1].copy()
        ylo, yhi, yempty = _x_extent_circle(Py, (bbox[1], bbox[0], bbox[3], bbox[2]))
        ok = empty | yempty | ((lo >= x0) & (hi <= x1 - 1) & (ylo >= y0) & (yhi <= y1 - 1))
        return t[ok]

    threads = threads or max(1, min(32, len(os.sched_getaffinity(0))))
    with ThreadPoolExecutor(threads) as pool:
        parts = list(pool.map(one, range(tiles * tiles)))
    # (the oracle's rows are canonical, and so are they in global ids: a tile's ids are
    # increasing; overlapping tiles give some rows more than once)
    acc = np.concatenate(parts).astype(np.int64)
    h = hull_count(xy)
    assert got.shape[0] == 2 * n - 2 - h, "%s: %d rows, Euler wants %d" % (what, got.shape[0], 2 * n - 2 - h)
    g64 = np.asarray(got, dtype=np.int64)
    missing = ~_members(acc, g64)
    assert not missing.any(), "%s: %d certified oracle triangles missing, e.g. %s" % (
        what, int(missing.sum()), acc[missing][:3].tolist())
    rest = got[~_members(g64, acc)]
    if rest.shape[0]:
        # the exact empty-circle test against every point near the circle: a float64
        # circumcircle widened by a margin above its rounding selects the candidates
        # (a k-d tree when SciPy is there), the exact SoS predicate decides
        P = x64[rest].astype(np.float64)
        ax, ay, bx, byy, cx, cy = P[:, 0, 0], P[:, 0, 1], P[:, 1, 0], P[:, 1, 1], P[:, 2, 0], P[:, 2, 1]
        d = 2.0 * (ax * (byy - cy) + bx * (cy - ay) + cx * (ay - byy))
        a2, b2, c2 = ax * ax + ay * ay, bx * bx + byy * byy, cx * cx + cy * cy
        ux = (a2 * (byy - cy) + b2 * (cy - ay) + c2 * (ay - byy)) / d
        uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d
        r = np.hypot(ax - ux, ay - uy) * (1 + 1e-9) + 2.0
        try:
            from scipy.spatial import cKDTree
            tree = cKDTree(x64.astype(np.float64))
            cands = tree.query_ball_point(np.stack([ux, uy], axis=1), r)
        except ImportError:
            by_x = np.argsort(x64[:, 0], kind="stable")
            xs = x64[by_x, 0]
            cands = []
            for k in range(rest.shape[0]):
                lo = np.searchsorted(xs, np.int64(np.floor(max(ux[k] - r[k], -2.0 ** 62))), "left")
                hi = np.searchsorted(xs, np.int64(np.ceil(min(ux[k] + r[k], 2.0 ** 62))), "right")
                c = by_x[lo:hi]
                c = c[(x64[c, 1] >= uy[k] - r[k]) & (x64[c, 1] <= uy[k] + r[k])]
                cands.append(c[(x64[c, 0] - ux[k]) ** 2 + (x64[c, 1] - uy[k]) ** 2 <= r[k] * r[k]])
        for k, tri in enumerate(rest):
            a, b, c = (int(v) for v in tri)
            bad = [int(q) for q in cands[k] if q not in (a, b, c) and oracle.incircle_sos(xy, a, b, c, int(q)) > 0]
            assert not bad, "%s: triangle %s has points %s in its circle" % (what, tri.tolist(), bad[:3])
    return acc.shape[0], rest.shape[0]


def _members(A, B):
    """For each row of A (int64, 3 columns): is it a row of B?  Rows are hashed
    (multiply-xor, wrapping 64-bit), B's hashes sorted, and every hash hit is confirmed
    by comparing the rows themselves."""
    def hsh(T):
        T = T.astype(np.uint64)
        return (T[:, 0] * np.uint64(0x9E3779B97F4A7C15)) ^ (T[:, 1] * np.uint64(0xC2B2AE3D27D4EB4F)) ^ \
               (T[:, 2] * np.uint64(0x165667B19E3779F9))
    if B.shape[0] == 0:
        return np.zeros(A.shape[0], dtype=bool)
    hb = hsh(B)
    o = np.argsort(hb, kind="stable")
    hb = hb[o]
    ha = hsh(A)
    pos = np.minimum(np.searchsorted(hb, ha), hb.shape[0] - 1)
    return (hb[pos] == ha) & (B[o[pos]] == A).all(axis=1)
