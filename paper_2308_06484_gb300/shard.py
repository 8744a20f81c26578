"""Strip sharding of one kinetic triangulation over several GPUs (one process per GPU).

The paper splits the plane into blocks that each own the points inside them; a point
that moves out of its block is sent to the block that now holds it (Section IV, Fig. 4),
and blocks only talk to their neighbours (Section V, Theorem 1).  Here the G x G
partitions are cut into `world` vertical strips of whole partition columns, one per rank:

- ownership: rank r owns the points whose current partition column lies in strip r;
- local set: rank r triangulates its owned points plus a halo, the points of the other
  strips whose x lies in [x_lo(r) - halo, x_hi(r) + halo) (the range the rank covers);
- exchange per step (the hand-off): every rank sends to every other rank the moves of
  its owned points whose old or new position lies in the receiver's covered range, so
  every rank knows every position it holds after the step; a point that leaves a strip
  is owned by the new strip's rank from then on;
- certificate: a triangle of rank r's triangulation is one of the whole set's when no
  point outside r's local set can lie in its circumcircle: the part of the circle inside
  the bounding box of all points (no point lies outside it) must have its x-range inside
  r's covered range; a hull edge a -> b of the local triangulation (the interior on its
  left) must be an edge of the whole set's hull (no vertex of that hull strictly right of
  it; the hull is gathered from every rank's local hull).  If every triangle and hull
  edge in the star of every owned point passes, each owned point's local star is its star
  in the whole triangulation; each rank then reports the triangles whose smallest id it
  owns, and their union is the whole triangulation, every triangle once.  If a test fails
  anywhere, every rank doubles the halo and collects its local set again.

Local ids are the local set's global ids in increasing order, so the tie-breaking of the
exact predicates (by id) decides exactly as for the whole set.  A local triangulation is
stepped kinetically while its set of points is unchanged and built again when points
enter or leave it.  The triangulator is passed in (a `Local`): the CUDA library on a GPU
(`KdtLocal`), anything with the same three methods elsewhere.

Exchange goes through torch.distributed (all_gather_object), gloo on CPU or NCCL; the
module has no kernel of its own.
"""
from __future__ import annotations

import numpy as np


class KdtLocal:
    """The local triangulator on this rank's GPU: a kdt handle."""

    def __init__(self, bits: int, device: int = 0, **cfg):
        self.bits, self.device, self.cfg = bits, device, cfg
        self.t = None

    def build(self, xy):
        from . import kdt
        if self.t is not None:
            self.t.close()
        self.t = kdt.Triangulation(kdt.default_config(domain_bits=self.bits, **self.cfg), device=self.device)
        self.t.build(np.ascontiguousarray(xy, dtype=np.int32))

    def step(self, moves):
        self.t.step(np.ascontiguousarray(moves, dtype=np.int32))

    def triangles(self):
        return self.t.export_triangles()

    def close(self):
        if self.t is not None:
            self.t.close()
            self.t = None


def _canonical(tris):
    """Rows rotated so the smallest id comes first (orientation kept), sorted."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    if t.shape[0] == 0:
        return t.astype(np.int32)
    r = np.argmin(t, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    t = np.take_along_axis(t, idx, axis=1)
    t = t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]
    return t.astype(np.int32)


def _x_extent_circle(P, bbox):
    """For triangles P (T, 3, 2) float64: the x-range [lo, hi] of circumcircle ∩ bbox,
    widened by a margin that covers the rounding of the float64 circumcentre, and
    whether that intersection is empty (then no point can lie in the circle)."""
    ax, ay = P[:, 0, 0], P[:, 0, 1]
    bx, by = P[:, 1, 0], P[:, 1, 1]
    cx, cy = P[:, 2, 0], P[:, 2, 1]
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    a2, b2, c2 = ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d
        uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d
        r = np.sqrt((ax - ux) ** 2 + (ay - uy) ** 2)
        x0, y0, x1, y1 = bbox
        margin = 1e-9 * (np.abs(ux) + np.abs(uy) + r) + 2.0
        # the widest chord of the circle inside the box's y-range
        dy = np.maximum(0.0, np.maximum(y0 - uy, uy - y1))
        hw = np.sqrt(np.maximum(0.0, r * r - dy * dy)) + margin
        lo = np.maximum(ux - hw, x0)
        hi = np.minimum(ux + hw, x1)
        finite = np.isfinite(ux) & np.isfinite(uy) & np.isfinite(r)
        empty = finite & ((dy > r + margin) | (lo > hi))
    return np.where(finite, lo, -np.inf), np.where(finite, hi, np.inf), empty


def _orient(a, b, c):
    """Exact orientation signs of rows (a, b, c) of int64 points (|coordinates| < 2^30)."""
    return np.sign((b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0]))


def _convex_hull(pts):
    """Strictly convex hull vertices of int64 points (monotone chain, exact)."""
    pts = np.unique(np.asarray(pts, dtype=np.int64).reshape(-1, 2), axis=0)
    if pts.shape[0] <= 2:
        return pts
    def chain(P):
        h = []
        for p in P:
            while len(h) >= 2 and (h[-1][0] - h[-2][0]) * (p[1] - h[-2][1]) - (h[-1][1] - h[-2][1]) * (p[0] - h[-2][0]) <= 0:
                h.pop()
            h.append(p)
        return h
    lower = chain(pts)
    upper = chain(pts[::-1])
    return np.array(lower[:-1] + upper[:-1], dtype=np.int64)


class StripShards:
    """This rank's strip of a sharded kinetic triangulation (see the module text).

    grid, bits: the G x G partitions of [0, 2^bits)^2; halo: initial halo width in
    coordinate units; local: this rank's triangulator (a `Local`); group: the process
    group (default: the world)."""

    def __init__(self, rank: int, world: int, grid: int, bits: int, halo: int, local, group=None):
        if grid < world:
            raise ValueError("need at least one partition column per rank")
        self.rank, self.world, self.grid, self.bits = rank, world, grid, bits
        self.halo = int(halo)
        self.local = local
        self.group = group
        self.ids = np.zeros(0, dtype=np.int64)      # local set: global ids, increasing
        self.xy = np.zeros((0, 2), dtype=np.int64)  # their positions
        self.bbox = None                            # of all points (float64 x0, y0, x1, y1)
        self.rebuilds = 0
        self.widenings = 0

    # ---- geometry of the strips
    def strip_x(self, r):
        """x-range [lo, hi) of strip r: partition columns c with c * world // G == r."""
        G, L = self.grid, 1 << self.bits
        cols = [c for c in range(G) if c * self.world // G == r]
        return (cols[0] * L) // G, -((-(cols[-1] + 1) * L) // G)

    def owner_of(self, x):
        col = (np.asarray(x, dtype=np.int64) * self.grid) >> self.bits
        return (col * self.world) // self.grid

    def covered(self, r, halo=None):
        h = self.halo if halo is None else halo
        lo, hi = self.strip_x(r)
        return lo - h, hi + h

    # ---- collectives
    def _all_gather(self, obj):
        import torch.distributed as dist
        out = [None] * self.world
        dist.all_gather_object(out, obj, group=self.group)
        return out

    def _any(self, flag: bool) -> bool:
        return any(self._all_gather(bool(flag)))

    # ---- set-up
    def start(self, ids, xy):
        """Take this rank's owned points from (ids, xy) (each rank passes its share, or
        all of them), collect the local sets and certify them (returns the widenings)."""
        ids = np.asarray(ids, dtype=np.int64)
        xy = np.asarray(xy, dtype=np.int64).reshape(-1, 2)
        own = self.owner_of(xy[:, 0]) == self.rank
        self._collect(ids[own], xy[own])
        return self.certify()

    def _collect(self, oid, oxy):
        """Local sets from every rank's owned points (oid, oxy of this rank), the bounding
        box of all points, then a fresh local triangulation."""
        parts = self._all_gather((oid, oxy))
        allmin = np.min([p[1].min(axis=0) for p in parts if p[1].shape[0]], axis=0)
        allmax = np.max([p[1].max(axis=0) for p in parts if p[1].shape[0]], axis=0)
        self.bbox = (float(allmin[0]), float(allmin[1]), float(allmax[0]), float(allmax[1]))
        lo, hi = self.covered(self.rank)
        ids, xy = [], []
        for pid, pxy in parts:
            keep = (pxy[:, 0] >= lo) & (pxy[:, 0] < hi)
            ids.append(pid[keep])
            xy.append(pxy[keep])
        ids = np.concatenate(ids)
        xy = np.concatenate(xy)
        o = np.argsort(ids, kind="stable")
        self.ids, self.xy = ids[o], xy[o]
        self._rebuild()

    def _rebuild(self):
        self.local.build(self.xy.astype(np.int32))
        self.rebuilds += 1

    def owned_mask(self):
        return self.owner_of(self.xy[:, 0]) == self.rank

    # ---- one time step
    def step(self, moves):
        """moves: (m, 3) rows (global id, x, y) of points this rank owns (rows for other
        points are ignored).  Exchange, update the local set, step or rebuild the local
        triangulation, certify (widening the halo until it holds).  Returns the number of
        halo widenings this step."""
        mv = np.asarray(moves, dtype=np.int64).reshape(-1, 3)
        pos = np.searchsorted(self.ids, mv[:, 0])
        pos = np.minimum(pos, max(0, self.ids.shape[0] - 1))
        mine = (self.ids.shape[0] > 0) & (self.ids[pos] == mv[:, 0])
        mine &= self.owner_of(self.xy[pos, 0]) == self.rank
        mv = mv[mine]
        old = self.xy[np.searchsorted(self.ids, mv[:, 0])] if mv.shape[0] else np.zeros((0, 2), np.int64)
        # the hand-off: to each rank the moves whose old or new position it covers
        out = []
        for s in range(self.world):
            lo, hi = self.covered(s)
            sel = ((old[:, 0] >= lo) & (old[:, 0] < hi)) | ((mv[:, 1] >= lo) & (mv[:, 1] < hi))
            out.append(mv[sel])
        got = self._all_gather(out)
        recv = np.concatenate([g[self.rank] for g in got]) if got else np.zeros((0, 3), np.int64)
        # positions after the step, within this rank's covered range
        lo, hi = self.covered(self.rank)
        rid = recv[:, 0]
        rpos = np.searchsorted(self.ids, rid)
        rpos_c = np.minimum(rpos, max(0, self.ids.shape[0] - 1))
        present = (self.ids.shape[0] > 0) & (self.ids[rpos_c] == rid)
        inside = (recv[:, 1] >= lo) & (recv[:, 1] < hi)
        leaving = present & ~inside
        entering = ~present & inside
        if leaving.any() or entering.any():
            keep = np.ones(self.ids.shape[0], dtype=bool)
            keep[rpos_c[leaving]] = False
            upd = present & inside
            xy = self.xy.copy()
            xy[rpos_c[upd]] = recv[upd, 1:]
            ids = np.concatenate([self.ids[keep], rid[entering]])
            xy = np.concatenate([xy[keep], recv[entering, 1:]])
            o = np.argsort(ids, kind="stable")
            self.ids, self.xy = ids[o], xy[o]
            self._rebuild()
        elif recv.shape[0]:
            loc = np.stack([rpos_c, recv[:, 1], recv[:, 2]], axis=1)
            self.xy[rpos_c] = recv[:, 1:]
            self.local.step(loc.astype(np.int32))
        # the bounding box of all points after the step
        bb = self._all_gather((self.xy.min(axis=0) if self.xy.shape[0] else None,
                               self.xy.max(axis=0) if self.xy.shape[0] else None))
        mins = [b[0] for b in bb if b[0] is not None]
        maxs = [b[1] for b in bb if b[1] is not None]
        self.bbox = (float(np.min([m[0] for m in mins])), float(np.min([m[1] for m in mins])),
                     float(np.max([m[0] for m in maxs])), float(np.max([m[1] for m in maxs])))
        return self.certify()

    # ---- certificate and output
    def _failures(self):
        """Triangles and hull edges in the stars of owned points that another rank's
        point could change: a triangle whose circumcircle, inside the bounding box of all
        points, reaches outside the covered x-range; a hull edge of the local set that is
        not one of the whole set (some vertex of the whole set's hull lies strictly right
        of it)."""
        tris = np.asarray(self.local.triangles(), dtype=np.int64).reshape(-1, 3)
        own = self.owned_mask()
        lo, hi = self.covered(self.rank)
        bad = 0
        star = own[tris].any(axis=1) if tris.shape[0] else np.zeros(0, dtype=bool)
        T = tris[star]
        if T.shape[0]:
            xlo, xhi, empty = _x_extent_circle(self.xy[T].astype(np.float64), self.bbox)
            bad += int(np.count_nonzero(~empty & ((xlo < lo) | (xhi > hi - 1))))
        # hull edges of the local triangulation: directed edges without a twin
        e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
        n = max(1, self.ids.shape[0])
        fwd = e[:, 0] * n + e[:, 1]
        rev = e[:, 1] * n + e[:, 0]
        hull = e[~np.isin(fwd, rev)]
        # the whole set's hull, from the union of every rank's local hull vertices
        verts = self.xy[np.unique(hull.ravel())] if hull.shape[0] else self.xy
        ghull = _convex_hull(np.concatenate(self._all_gather(verts)))
        hull = hull[own[hull].any(axis=1)]
        if hull.shape[0] and ghull.shape[0] >= 3:
            A = self.xy[hull[:, 0]][:, None, :]
            B = self.xy[hull[:, 1]][:, None, :]
            right = _orient(A, B, ghull[None, :, :]) < 0
            bad += int(np.count_nonzero(right.any(axis=1)))
        return bad

    def certify(self):
        """Widen the halo (x 2, collecting every local set again) until every rank's
        certificate holds; returns the number of widenings."""
        widen = 0
        while self._any(self._failures() > 0):
            self.halo *= 2
            widen += 1
            self.widenings += 1
            own = self.owned_mask()
            self._collect(self.ids[own], self.xy[own])
            if self.halo > (4 << self.bits):
                raise RuntimeError("halo covers the whole domain and the certificate still fails")
        return widen

    def owned_triangles(self):
        """This rank's share of the whole triangulation: triangles whose smallest global
        id it owns, in global ids, canonical (rotated, sorted)."""
        tris = np.asarray(self.local.triangles(), dtype=np.int64).reshape(-1, 3)
        g = self.ids[tris]
        first = np.argmin(g, axis=1)
        own = self.owned_mask()
        mine = own[tris[np.arange(tris.shape[0]), first]]
        return _canonical(g[mine])

    def gather_triangles(self):
        """The whole triangulation on every rank (canonical), from every rank's share."""
        parts = self._all_gather(self.owned_triangles())
        return _canonical(np.concatenate(parts))
