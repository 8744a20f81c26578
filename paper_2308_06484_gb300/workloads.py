"""Seeded synthetic workloads for the kinetic Delaunay update.

This module only draws inputs: point sets and per-step move lists.  It holds none
of the method's arithmetic (no predicate, no triangulation) and is shared by the
CUDA path's tests and benchmark and by the oracle's tests.

The paper (Section III, "movepoint_i"; Fig. 4) moves one randomly chosen point
per block per time step, each move going right, left, up or down (Lemma 1).  The
workloads follow that statement with the sizes used to exercise the method:

========  =============================================================  ======  ==============
name      points                                                          grid    moves / cell
========  =============================================================  ======  ==============
c1        1,000 uniform on [0, 2^16)^2, seed 1                            4x4     1, 1 unit
c2        1,000,000 uniform on [0, 2^24)^2                                64x64   1, 1-8 units
c3        16,000,000: 32-Gaussian mixture (sigma 2^18) + 5 % lattice      256^2   1-16, 1-8 units
c4        512 instances, n_i log-uniform in [1e3, 2e5], on [0, 2^20)^2    ~256/c  1-4, 1-8 units
========  =============================================================  ======  ==============

Move rule (the same for every workload): for every cell in row-major order, the
requested number of distinct points currently in that cell is chosen at random;
each draws a direction (R/L/U/D) and a distance.  A target is rejected and
redrawn (at most 64 times, else that slot is skipped) if it leaves [0, 2^B)^2,
coincides with any position held at the start of the step, or coincides with a
target already accepted in this step.  Final positions are therefore distinct and
no target lands on a position vacated in the same step.
"""
from __future__ import annotations

import math

import numpy as np

DIRS = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]], dtype=np.int64)  # R, L, U, D


def _key(xy):
    xy = np.asarray(xy, dtype=np.int64)
    return (xy[..., 0] << 32) | xy[..., 1]


def uniform_points(n: int, bits: int, seed: int) -> np.ndarray:
    """n distinct integer points uniform on [0, 2^bits)^2 (int32, shape (n, 2))."""
    rng = np.random.default_rng(seed)
    have = np.empty((0, 2), dtype=np.int64)
    while have.shape[0] < n:
        need = n - have.shape[0]
        cand = rng.integers(0, 1 << bits, size=(need + need // 8 + 16, 2), dtype=np.int64)
        allp = np.concatenate([have, cand])
        _, first = np.unique(_key(allp), return_index=True)
        first.sort()
        have = allp[first]
    have = have[:n]
    return np.ascontiguousarray(have.astype(np.int32))


def mixture_lattice_points(n: int, bits: int, seed: int, n_comp: int = 32,
                           sigma: float = float(1 << 18), lattice_frac: float = 0.05,
                           patches: int = 8, spacing: int = 64) -> np.ndarray:
    """Gaussian-mixture points plus an exact integer lattice (cocircular 2x2 cells).

    Lattice: ``patches`` square patches of side ceil(sqrt(n_lat / patches)) nodes,
    spacing ``spacing``, each at a seeded random origin, the last one trimmed so
    that exactly n_lat = round(lattice_frac * n) lattice points exist.  Mixture:
    equal weights, centres uniform on the domain, samples drawn in double and
    rounded to nearest (ties to even), rejected outside the domain or on an
    occupied position.  Ids: lattice points first, then mixture points, then the
    whole set is shuffled with the same seed.
    """
    rng = np.random.default_rng(seed)
    L = 1 << bits
    n_lat = int(round(lattice_frac * n))
    side = int(math.ceil(math.sqrt(n_lat / patches))) if n_lat else 0
    lat = []
    left = n_lat
    for p in range(patches):
        if left <= 0:
            break
        ext = (side - 1) * spacing
        ox, oy = rng.integers(0, L - ext, size=2)
        gx, gy = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
        pts = np.stack([ox + gx.ravel() * spacing, oy + gy.ravel() * spacing], axis=1)
        lat.append(pts[:left])
        left -= pts[:left].shape[0]
    lat = np.concatenate(lat).astype(np.int64) if lat else np.empty((0, 2), np.int64)
    _, first = np.unique(_key(lat), return_index=True)
    first.sort()
    lat = lat[first]
    centres = rng.random((n_comp, 2)) * L
    have = lat
    while have.shape[0] < n:
        need = n - have.shape[0]
        m = need + need // 16 + 64
        comp = rng.integers(0, n_comp, size=m)
        s = centres[comp] + rng.standard_normal((m, 2)) * sigma
        s = np.rint(s)
        ok = np.all((s >= 0) & (s < L), axis=1)
        s = s[ok].astype(np.int64)
        allp = np.concatenate([have, s])
        _, first = np.unique(_key(allp), return_index=True)
        first.sort()
        have = allp[first]
    have = have[:n]
    perm = rng.permutation(n)
    return np.ascontiguousarray(have[perm].astype(np.int32))


def cell_of(xy, grid: int, bits: int) -> np.ndarray:
    """Row-major cell index of each point in the grid x grid equal-area partition."""
    xy = np.asarray(xy, dtype=np.int64)
    cx = (xy[:, 0] * grid) >> bits
    cy = (xy[:, 1] * grid) >> bits
    return cy * grid + cx


def _stable_order(cells, ncell):
    """Indices sorting `cells` stably (a radix sort when the cell index fits 16 bits)."""
    if ncell <= 65536:
        return np.argsort(cells.astype(np.uint16), kind="stable")
    return np.argsort(cells, kind="stable")


class KineticWorkload:
    """A point set plus a seeded stream of per-step moves.

    ``next_moves()`` returns an (m, 3) int32 array of (id, new_x, new_y) and
    advances the positions.  ``positions`` is the current (n, 2) int32 array.
    """

    def __init__(self, xy, grid: int, bits: int, moves_per_cell=(1, 1),
                 dist=(1, 1), seed: int = 0, name: str = ""):
        self.name = name
        self.grid = int(grid)
        self.bits = int(bits)
        self.mpc = (int(moves_per_cell[0]), int(moves_per_cell[1]))
        self.dist = (int(dist[0]), int(dist[1]))
        self.rng = np.random.default_rng(seed)
        self.pos = np.ascontiguousarray(np.asarray(xy, dtype=np.int64).reshape(-1, 2))
        self.skeys = np.sort(_key(self.pos))
        self.cells = cell_of(self.pos, self.grid, self.bits)  # kept current for moved points
        self.step_index = 0

    @property
    def n(self):
        return self.pos.shape[0]

    @property
    def positions(self):
        return np.ascontiguousarray(self.pos.astype(np.int32))

    def _choose(self):
        G = self.grid
        cells = self.cells
        counts = np.bincount(cells, minlength=G * G)
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        lo, hi = self.mpc
        want = self.rng.integers(lo, hi + 1, size=G * G)
        want = np.minimum(want, counts)
        if hi == 1:
            order = _stable_order(cells, G * G)
            cs = np.nonzero(want)[0]
            off = (self.rng.random(cs.shape[0]) * counts[cs]).astype(np.int64)
            chosen = order[starts[cs] + off]
            return chosen
        # several points per cell: random keys; per cell the `want` points with the
        # smallest keys (ties by id), in (cell, key, id) order
        rk = self.rng.random(self.n)
        # Only keys below a per-cell threshold can be among the smallest `want` as long
        # as at least `want` keys of that cell are below it; cells short of that keep
        # every point.  The selection is the same as sorting every point.
        thr = (want + 4.0 * np.sqrt(want) + 8.0) / np.maximum(counts, 1)
        cand = rk < thr[cells]
        short = np.bincount(cells[cand], minlength=G * G) < want
        if short.any():
            cand |= short[cells]
        idx = np.nonzero(cand)[0]
        o = np.lexsort((rk[idx], cells[idx]))  # stable: ties keep increasing id
        order2 = idx[o]
        c_o = cells[order2]
        cstart = np.concatenate([[0], np.cumsum(np.bincount(c_o, minlength=G * G))[:-1]])
        rank = np.arange(order2.shape[0]) - cstart[c_o]
        sel = rank < want[c_o]
        return order2[sel]

    def next_moves(self) -> np.ndarray:
        ids = self._choose()
        m = ids.shape[0]
        L = 1 << self.bits
        tx = np.empty(m, dtype=np.int64)
        ty = np.empty(m, dtype=np.int64)
        accepted = np.zeros(m, dtype=bool)
        acc_keys = np.empty(0, dtype=np.int64)
        pending = np.arange(m)
        for _ in range(64):
            if pending.size == 0:
                break
            d = self.rng.integers(0, 4, size=pending.size)
            s = self.rng.integers(self.dist[0], self.dist[1] + 1, size=pending.size)
            nx = self.pos[ids[pending], 0] + DIRS[d, 0] * s
            ny = self.pos[ids[pending], 1] + DIRS[d, 1] * s
            ok = (nx >= 0) & (nx < L) & (ny >= 0) & (ny < L)
            k = (nx << 32) | ny
            idx = np.searchsorted(self.skeys, k)
            idx = np.minimum(idx, self.skeys.size - 1)
            ok &= self.skeys[idx] != k
            if acc_keys.size:
                j = np.searchsorted(acc_keys, k)
                j = np.minimum(j, acc_keys.size - 1)
                ok &= acc_keys[j] != k
            # among this round's candidates the first (in cell, slot order) wins
            cand = np.nonzero(ok)[0]
            if cand.size:
                _, first = np.unique(k[cand], return_index=True)
                win = cand[np.sort(first)]
                tx[pending[win]] = nx[win]
                ty[pending[win]] = ny[win]
                accepted[pending[win]] = True
                acc_keys = np.sort(np.concatenate([acc_keys, k[win]]))
            keep = np.ones(pending.size, dtype=bool)
            if cand.size:
                keep[win] = False
            pending = pending[keep]
        sel = np.nonzero(accepted)[0]
        ids = ids[sel]
        moves = np.stack([ids, tx[sel], ty[sel]], axis=1).astype(np.int32)
        # advance positions and the occupancy index
        old = _key(self.pos[ids])
        self.pos[ids, 0] = tx[sel]
        self.pos[ids, 1] = ty[sel]
        self.cells[ids] = cell_of(self.pos[ids], self.grid, self.bits)
        new = _key(self.pos[ids])
        keep = np.ones(self.skeys.size, dtype=bool)
        keep[np.searchsorted(self.skeys, old)] = False
        rest = self.skeys[keep]
        new = np.sort(new)
        self.skeys = np.insert(rest, np.searchsorted(rest, new), new)
        self.step_index += 1
        return np.ascontiguousarray(moves)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def c1(seed: int = 1) -> KineticWorkload:
    """1,000 uniform points on [0,2^16)^2, 4x4 cells, one 1-unit move per cell."""
    return KineticWorkload(uniform_points(1000, 16, seed), grid=4, bits=16,
                           moves_per_cell=(1, 1), dist=(1, 1), seed=seed + 1000, name="c1")


def c2(n: int = 1_000_000, grid: int = 64, seed: int = 2) -> KineticWorkload:
    """1e6 uniform points on [0,2^24)^2, 64x64 cells, one 1-8 unit move per cell."""
    return KineticWorkload(uniform_points(n, 24, seed), grid=grid, bits=24,
                           moves_per_cell=(1, 1), dist=(1, 8), seed=seed + 1000, name="c2")


def c3(n: int = 16_000_000, grid: int = 256, seed: int = 3) -> KineticWorkload:
    """Gaussian mixture + 5 % lattice, 256x256 cells, 1-16 moves of 1-8 units per cell."""
    return KineticWorkload(mixture_lattice_points(n, 24, seed), grid=grid, bits=24,
                           moves_per_cell=(1, 16), dist=(1, 8), seed=seed + 1000, name="c3")


def c4_sizes(n_inst: int = 512, seed: int = 4, lo: float = 1e3, hi: float = 2e5):
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_inst))).astype(np.int64)


def c4_grid(n_i: int) -> int:
    """Cells per side so that a cell holds about 256 points."""
    return max(1, int(round(math.sqrt(n_i / 256.0))))


def c4(n_inst: int = 512, seed: int = 4, lo: float = 1e3, hi: float = 2e5):
    """512 independent instances on [0,2^20)^2, ~256 points per cell, 1-4 moves per cell."""
    sizes = c4_sizes(n_inst, seed, lo, hi)
    out = []
    for i, n_i in enumerate(sizes):
        xy = uniform_points(int(n_i), 20, seed * 100003 + i)
        out.append(KineticWorkload(xy, grid=c4_grid(int(n_i)), bits=20, moves_per_cell=(1, 4),
                                   dist=(1, 8), seed=seed * 7919 + i, name="c4[%d]" % i))
    return out
