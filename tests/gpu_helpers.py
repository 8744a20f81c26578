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
    """Points on the convex hull boundary, collinear ones included (monotone chain)."""
    pts = np.unique(np.asarray(xy, dtype=np.int64), axis=0)
    if pts.shape[0] < 3:
        return pts.shape[0]

    def chain(P):
        h = []
        for p in P:
            while len(h) >= 2 and (h[-1][0] - h[-2][0]) * (p[1] - h[-2][1]) - (h[-1][1] - h[-2][1]) * (p[0] - h[-2][0]) < 0:
                h.pop()
            h.append((int(p[0]), int(p[1])))
        return h
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
    from paper_2308_06484_gb300.shard import _x_extent_circle, _canonical
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
    acc = _canonical(np.unique(_canonical(np.concatenate(parts)), axis=0))
    h = hull_count(xy)
    assert got.shape[0] == 2 * n - 2 - h, "%s: %d rows, Euler wants %d" % (what, got.shape[0], 2 * n - 2 - h)
    key = lambda t: (t[:, 0].astype(np.int64) * n + t[:, 1]) * n + t[:, 2]
    kg, ka = key(got.astype(np.int64)), key(acc.astype(np.int64))
    missing = ~np.isin(ka, kg)
    assert not missing.any(), "%s: %d certified oracle triangles missing, e.g. %s" % (
        what, int(missing.sum()), acc[missing][:3].tolist())
    rest = got[~np.isin(kg, ka)]
    for tri in rest:
        a, b, c = (int(v) for v in tri)
        P = x64[[a, b, c]].astype(np.float64)
        d = 2.0 * (P[0, 0] * (P[1, 1] - P[2, 1]) + P[1, 0] * (P[2, 1] - P[0, 1]) + P[2, 0] * (P[0, 1] - P[1, 1]))
        s = (P ** 2).sum(axis=1)
        ux = (s[0] * (P[1, 1] - P[2, 1]) + s[1] * (P[2, 1] - P[0, 1]) + s[2] * (P[0, 1] - P[1, 1])) / d
        uy = (s[0] * (P[2, 0] - P[1, 0]) + s[1] * (P[0, 0] - P[2, 0]) + s[2] * (P[1, 0] - P[0, 0])) / d
        r = np.hypot(P[0, 0] - ux, P[0, 1] - uy) * (1 + 1e-9) + 2.0
        cand = np.nonzero((x64[:, 0] >= ux - r) & (x64[:, 0] <= ux + r) & (x64[:, 1] >= uy - r) &
                          (x64[:, 1] <= uy + r))[0]
        bad = [int(q) for q in cand if q not in (a, b, c) and oracle.incircle_sos(xy, a, b, c, int(q)) > 0]
        assert not bad, "%s: triangle %s has points %s in its circle" % (what, tri.tolist(), bad[:3])
    return acc.shape[0], rest.shape[0]
