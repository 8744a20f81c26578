"""Independent mathematical pins for the oracle (pure Python / numpy).

Nothing here calls the oracle or the CUDA library.  These are the closed forms and
brute-force definitions the oracle's results are checked against:

- ``det4_lifted``: the 4x4 determinant of the lifted rows (x, y, x^2+y^2, 1),
  expanded by cofactors in exact Python integers (a different formula from the
  oracle's translated 3x3 form).
- ``sos_incircle_bigint``: the Simulation-of-Simplicity sign obtained by
  *evaluating* the perturbed determinant with concrete integer weights
  z_i = S*(x_i^2+y_i^2) + W^(3-rank_i), S >> W^3 * (cofactor bound); no cofactor
  rule is written out.
- ``brute_force_dt``: every counter-clockwise non-degenerate triple whose
  circumcircle (SoS) contains no other point (Section I definition).
- ``hull_boundary``: the convex hull boundary with collinear points, by the
  monotone chain, as directed ccw edges.
"""
from __future__ import annotations

import itertools

import numpy as np


def det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def det4(m):
    tot = 0
    for j in range(4):
        minor = [[m[i][k] for k in range(4) if k != j] for i in range(1, 4)]
        tot += (-1) ** j * m[0][j] * det3(minor)
    return tot


def orient_bigint(p, q, r):
    """det [[px,py,1],[qx,qy,1],[rx,ry,1]] in exact integers."""
    return det3([[int(p[0]), int(p[1]), 1], [int(q[0]), int(q[1]), 1], [int(r[0]), int(r[1]), 1]])


def det4_lifted(pts):
    rows = [[int(x), int(y), int(x) * int(x) + int(y) * int(y), 1] for x, y in pts]
    return det4(rows)


def sign(v):
    return (v > 0) - (v < 0)


def sos_incircle_bigint(xy, a, b, c, d):
    """Sign of the perturbed lifted determinant with rows a, b, c, d.

    The perturbation of point i is eps^(rank of i), with a smaller id having the
    larger perturbation.  It is realised exactly by scaling the true lift by S and
    adding W^(3 - rank): the unperturbed term dominates whenever it is non-zero
    (|D| >= 1 so |S*D| >= S), and each weight dominates all smaller ones.
    """
    ids = [a, b, c, d]
    rank = {v: r for r, v in enumerate(sorted(ids))}
    W = 1 << 130   # > 2 * 4 * max |cofactor| (cofactors < 2^60 for 28-bit inputs)
    S = 1 << 600   # > 4 * W^3 * max |cofactor|
    rows = []
    for v in ids:
        x, y = int(xy[v][0]), int(xy[v][1])
        rows.append([x, y, S * (x * x + y * y) + W ** (3 - rank[v]), 1])
    return sign(det4(rows))


def brute_force_dt(xy):
    """Canonical DT by the empty-circumcircle definition (Section I), SoS ties.

    O(n^4); use for n <= ~40 and coordinates < 2^12.  The raw determinant and
    the ties are both evaluated in exact Python integers.
    """
    xy = np.asarray(xy, dtype=np.int64)
    n = xy.shape[0]
    assert np.abs(xy).max() < (1 << 12)
    X = xy[:, 0]
    Y = xy[:, 1]
    Z = X * X + Y * Y
    out = []
    for a, b, c in itertools.combinations(range(n), 3):
        o = orient_bigint(xy[a], xy[b], xy[c])
        if o == 0:
            continue
        if o < 0:
            b, c = c, b
        # raw lifted 4x4 determinant for all other points d (exact, object ints)
        others = [d for d in range(n) if d not in (a, b, c)]
        if not others:
            out.append((a, b, c))
            continue
        dd = np.array(others)
        rows = [[int(X[v]), int(Y[v]), int(Z[v]), 1] for v in (a, b, c)]
        rows.append([X[dd].astype(object), Y[dd].astype(object), Z[dd].astype(object), 1])
        D = det4(rows)
        ok = True
        for k, d in enumerate(others):
            s = sign(D[k]) if D[k] != 0 else sos_incircle_bigint(xy, a, b, c, int(d))
            if s > 0:
                ok = False
                break
        if ok:
            out.append((a, b, c))
    canon = []
    for t in out:
        r = int(np.argmin(t))
        canon.append(tuple(int(v) for v in (t[r:] + t[:r])))
    return sorted(canon)


def hull_boundary(xy):
    """Directed ccw boundary edges of the convex hull, collinear points kept.

    Strict hull by Andrew's monotone chain, then every input point lying on a
    strict hull edge is inserted in order along that edge.
    """
    xy = np.asarray(xy, dtype=np.int64)
    pts = sorted(range(xy.shape[0]), key=lambda i: (int(xy[i, 0]), int(xy[i, 1])))

    def cross(o, a, b):
        return orient_bigint(xy[o], xy[a], xy[b])

    lower, upper = [], []
    for i in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], i) <= 0:
            lower.pop()
        lower.append(i)
    for i in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], i) <= 0:
            upper.pop()
        upper.append(i)
    strict = lower[:-1] + upper[:-1]
    edges = []
    h = len(strict)
    for k in range(h):
        u, v = strict[k], strict[(k + 1) % h]
        on = []
        for w in range(xy.shape[0]):
            if w in (u, v):
                continue
            if cross(u, v, w) == 0:
                d1 = int(np.dot(xy[w] - xy[u], xy[v] - xy[u]))
                d2 = int(np.dot(xy[w] - xy[v], xy[u] - xy[v]))
                if d1 > 0 and d2 > 0:
                    on.append((d1, w))
        chain = [u] + [w for _, w in sorted(on)] + [v]
        edges.extend(zip(chain[:-1], chain[1:]))
    return sorted(edges)


def boundary_edges_of(tris):
    """Directed edges used by exactly one triangle (the hull, traversed ccw)."""
    seen = set()
    for a, b, c in np.asarray(tris).tolist():
        seen.update([(a, b), (b, c), (c, a)])
    return sorted((a, b) for (a, b) in seen if (b, a) not in seen)
