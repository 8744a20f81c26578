"""CPU reference of the proposal's training rows — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
this module.  It shares no code with the CUDA path.

A row describes one move of point p from its position to q (paper, Fig. 4: delete
the moved point, update its position, insert it again), taken on the triangulation
DT(P) in force when the move starts.  The definitions are the ones ``include/kdt.h``
states; here they are computed from whole triangulations built by the oracle:

* link: the neighbours v_0..v_{k-1} of p in DT(P), counter-clockwise (p interior).
* start j0: the one j whose half-open wedge [dir(v_j), dir(v_{j+1})) around p holds
  the move direction d = q - p (exact integer cross products).  Rotated index
  r(v_j) = (j - j0) mod k.
* hole triangles: the k - 2 triangles of DT(P \\ {p}) that DT(P) does not have (the
  re-triangulated hole of the deletion).  Each is named by its rotated vertex
  indices sorted ascending; the names sorted lexicographically give the ranks.
* slot: the smallest rank of a hole triangle whose closed region holds q; 16
  ("beyond") when none does or that rank is 16 or more.
* conflict size: the number of triangles of DT(P \\ {p}) that DT(P') lacks, P' = P
  with p at q (the cavity of the insertion).
* features (float32): f0 = |d| / R, f1 = k / 16, and for r = 0..14 the vertex of
  rotated index r relative to p in the frame (u, n) of the move, u = d / |d|,
  n = u turned a quarter ccw, divided by R: f[2+2r] = <v - p, u> / R,
  f[3+2r] = <v - p, n> / R (0 where r >= k).  R = mean |v_j - p|.
"""
from __future__ import annotations

import numpy as np

import oracle

BEYOND = 16
N_FEAT = 32


def _orient(a, b, c):
    return (int(b[0]) - int(a[0])) * (int(c[1]) - int(a[1])) - (int(b[1]) - int(a[1])) * (int(c[0]) - int(a[0]))


def _tri_set(tris):
    return set(map(tuple, np.asarray(tris).tolist()))


def link_ccw(tris, p):
    """Counter-clockwise link of p from a canonical triangle list, None if p is on the hull."""
    nxt = {}
    for t in np.asarray(tris).tolist():
        if p in t:
            i = t.index(p)
            a, b = t[(i + 1) % 3], t[(i + 2) % 3]
            nxt[a] = b
    if not nxt:
        return None
    # interior iff every link vertex has a successor and a predecessor (a closed cycle)
    if set(nxt.keys()) != set(nxt.values()):
        return None
    start = min(nxt)
    out = [start]
    while True:
        v = nxt[out[-1]]
        if v == start:
            break
        out.append(v)
    if len(out) != len(nxt):
        return None
    return out


def wedge_start(xy, p, link, d):
    """Index j0 of the wedge [dir v_j, dir v_{j+1}) holding direction d (exactly one)."""
    P = xy[p]
    k = len(link)
    hits = []
    for j in range(k):
        a = (int(xy[link[j]][0]) - int(P[0]), int(xy[link[j]][1]) - int(P[1]))
        b = (int(xy[link[(j + 1) % k]][0]) - int(P[0]), int(xy[link[(j + 1) % k]][1]) - int(P[1]))
        c1 = a[0] * d[1] - a[1] * d[0]      # cross(a, d)
        c2 = d[0] * b[1] - d[1] * b[0]      # cross(d, b)
        if c1 >= 0 and c2 > 0:
            hits.append(j)
    if len(hits) != 1:
        raise ValueError("direction is not in exactly one wedge: %r" % hits)
    return hits[0]


def features(xy, p, q, link, j0):
    """The 32 float32 features of moving p to q (link and j0 as above)."""
    xy = np.asarray(xy)
    k = len(link)
    P = xy[p].astype(np.int64)
    d = np.asarray(q, dtype=np.int64) - P
    f32 = np.float32
    dx, dy = f32(d[0]), f32(d[1])
    s = np.sqrt(f32(dx * dx + dy * dy))
    ux, uy = f32(dx / s), f32(dy / s)
    rel = [(f32(int(xy[v][0]) - int(P[0])), f32(int(xy[v][1]) - int(P[1]))) for v in link]
    R = f32(0)
    for r in range(k):  # summed in rotated order, starting at j0
        rx, ry = rel[(j0 + r) % k]
        R = f32(R + np.sqrt(f32(rx * rx + ry * ry)))
    R = f32(R / f32(k))
    f = np.zeros(N_FEAT, dtype=np.float32)
    f[0] = s / R
    f[1] = f32(k) / f32(16)
    for r in range(min(k, 15)):
        rx, ry = rel[(j0 + r) % k]
        f[2 + 2 * r] = f32(rx * ux + ry * uy) / R
        f[3 + 2 * r] = f32(ry * ux - rx * uy) / R
    return f


def without(xy, p):
    """DT(P \\ {p}) as a canonical list in the original ids (ids above p shift back)."""
    xy = np.asarray(xy, dtype=np.int32)
    rest = np.delete(xy, p, axis=0)
    t = oracle.delaunay(rest).astype(np.int64)
    t[t >= p] += 1
    return t


def row(xy, p, q):
    """(features, slot, conflict size) of moving p to q, or None if p is on the hull.

    Three oracle triangulations: DT(P), DT(P \\ {p}), DT(P')."""
    xy = np.asarray(xy, dtype=np.int32)
    T0 = oracle.delaunay(xy)
    link = link_ccw(T0, p)
    if link is None:
        return None
    k = len(link)
    d = (int(q[0]) - int(xy[p][0]), int(q[1]) - int(xy[p][1]))
    j0 = wedge_start(xy, p, link, d)
    rot = {v: (j - j0) % k for j, v in enumerate(link)}
    T1 = without(xy, p)
    hole = sorted(_tri_set(T1) - _tri_set(T0))
    named = sorted((tuple(sorted(rot[v] for v in t)), t) for t in hole)
    slot = BEYOND
    for rank, (_, t) in enumerate(named):
        a, b, c = xy[t[0]], xy[t[1]], xy[t[2]]
        if _orient(a, b, q) >= 0 and _orient(b, c, q) >= 0 and _orient(c, a, q) >= 0:
            slot = rank if rank < BEYOND else BEYOND
            break
    xy2 = xy.copy()
    xy2[p] = q
    T2 = oracle.delaunay(xy2)
    conflict = len(_tri_set(T1) - _tri_set(T2))
    return features(xy, p, q, link, j0), slot, conflict, {"link": link, "j0": j0, "hole": named, "T1": T1, "T2": T2}
