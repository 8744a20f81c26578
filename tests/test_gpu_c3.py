"""The 16e6-point workload (Gaussian mixture + 5 % lattice, 256x256 partitions, 1-16
moves per partition) at full size.  The oracle cannot triangulate 1.6e7 points in a
test's time, so the result is checked by properties that fix it at any size: the
oracle's certifier (every triangle counter-clockwise, every edge shared by two
triangles, the boundary winding once, Euler's count, every interior edge locally
Delaunay with the SoS predicate: together the definition of the unique triangulation),
and, on sampled triangles, the empty-circle definition itself against every point with
the oracle's exact predicate (including lattice triangles, whose circles pass through
other lattice points and are decided by SoS)."""
import numpy as np
import pytest

import oracle
from paper_2308_06484_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _empty_circle(xy, tri):
    """No point strictly inside the (SoS) circumcircle of tri, checked exactly on every
    point of the circle's bounding box (float64 box with a margin)."""
    a, b, c = (int(v) for v in tri)
    P = xy[[a, b, c]].astype(np.float64)
    ax, ay = P[0]
    bx, by = P[1]
    cx, cy = P[2]
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
    r = np.hypot(ax - ux, ay - uy) * (1 + 1e-9) + 2.0
    m = (xy[:, 0] >= ux - r) & (xy[:, 0] <= ux + r) & (xy[:, 1] >= uy - r) & (xy[:, 1] <= uy + r)
    cand = np.nonzero(m)[0]
    bad = [int(q) for q in cand if q not in (a, b, c) and oracle.incircle_sos(xy, a, b, c, int(q)) > 0]
    return bad, len(cand)


def test_c3_full_size():
    import torch
    from paper_2308_06484_gb300 import kdt
    w = W.c3()
    t = kdt.Triangulation(kdt.default_config(grid=256, domain_bits=24))
    t.build(torch.from_numpy(w.positions).cuda())
    assert t.verify() == 0
    moved = 0
    for _ in range(2):
        mv = w.next_moves()
        moved += mv.shape[0]
        t.step(torch.from_numpy(mv).cuda())
    assert moved > 100000
    assert t.verify() == 0
    xy = w.positions
    assert np.array_equal(t.export_points(), xy)
    tris = t.export_triangles()
    assert tris.shape[0] > 2 * xy.shape[0] - 2 - 100000
    assert oracle.check_dt(xy, tris) == 0
    rng = np.random.default_rng(7)
    sample = list(rng.choice(tris.shape[0], 24, replace=False))
    # lattice triangles: an axis-aligned edge of exactly one lattice spacing
    e = xy[tris[:, 1]].astype(np.int64) - xy[tris[:, 0]].astype(np.int64)
    lat = np.nonzero(((np.abs(e[:, 0]) == 64) & (e[:, 1] == 0)) | ((e[:, 0] == 0) & (np.abs(e[:, 1]) == 64)))[0]
    assert lat.size > 1000
    sample += list(rng.choice(lat, 16, replace=False))
    for i in sample:
        bad, n = _empty_circle(xy, tris[i])
        assert not bad, (tris[i], bad[:3])
    st = t.stats()
    assert st["fallbacks"] == 0
