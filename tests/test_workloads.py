"""The seeded generators produce what the workload descriptions say (no GPU)."""
import numpy as np

from paper_2308_06484_gb300 import workloads as W


def _check_steps(w, steps, per_cell, dist):
    G, B = w.grid, w.bits
    for _ in range(steps):
        before = w.positions.astype(np.int64)
        cells = W.cell_of(before, G, B)
        occupied = set(map(tuple, before.tolist()))
        m = w.next_moves().astype(np.int64)
        after = w.positions.astype(np.int64)
        ids = m[:, 0]
        assert len(np.unique(ids)) == len(ids)
        d = m[:, 1:] - before[ids]
        # axis-aligned moves (Lemma 1) of the allowed length
        assert np.all((d[:, 0] == 0) | (d[:, 1] == 0))
        L = np.abs(d).sum(axis=1)
        assert np.all((L >= dist[0]) & (L <= dist[1]))
        assert np.all((m[:, 1:] >= 0) & (m[:, 1:] < (1 << B)))
        for x, y in m[:, 1:].tolist():
            assert (x, y) not in occupied
        assert len(np.unique(after[:, 0] << 32 | after[:, 1])) == w.n
        cnt = np.bincount(cells[ids], minlength=G * G)
        assert cnt.max() <= per_cell[1]
        occupied_cells = np.bincount(cells, minlength=G * G) > 0
        # almost every non-empty cell moves at least per_cell[0] points
        assert np.mean(cnt[occupied_cells] >= per_cell[0]) > 0.95
        assert np.array_equal(after[ids], m[:, 1:])


def test_c1():
    w = W.c1()
    assert w.n == 1000 and w.grid == 4 and w.bits == 16
    xy = w.positions
    assert xy.min() >= 0 and xy.max() < (1 << 16)
    _check_steps(w, 20, (1, 1), (1, 1))


def test_c2_shaped_small():
    w = W.c2(n=20000, grid=16)
    _check_steps(w, 5, (1, 1), (1, 8))


def test_multi_move_cells():
    w = W.KineticWorkload(W.uniform_points(20000, 24, 5), 16, 24, (1, 16), (1, 8), seed=3)
    _check_steps(w, 4, (1, 16), (1, 8))


def test_mixture_lattice():
    xy = W.mixture_lattice_points(40000, 24, 7)
    assert xy.shape == (40000, 2)
    assert len(np.unique(xy.astype(np.int64)[:, 0] << 32 | xy[:, 1])) == 40000
    # the lattice part holds unit cells of spacing 64 (cocircular quadruples)
    s = set(map(tuple, xy.tolist()))
    quads = sum(1 for (x, y) in list(s)[:20000]
                if (x + 64, y) in s and (x, y + 64) in s and (x + 64, y + 64) in s)
    assert quads > 100


def test_determinism():
    a = W.c1().next_moves()
    b = W.c1().next_moves()
    assert np.array_equal(a, b)


def test_c4_sizes():
    s = W.c4_sizes()
    assert s.shape == (512,)
    assert s.min() >= 1000 and s.max() <= 200000
    assert 2.5e7 > s.sum() > 1.2e7   # E = 512 * (2e5 - 1e3) / ln 200 = 1.92e7
