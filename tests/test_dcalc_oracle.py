"""Pins for the d-calculation reference (no GPU): closed forms on a square lattice
(interior, edge and corner points differ, so an off-by-one in N fails), a hand
example, SciPy's k-d tree (a library routine for the same query), monotonicity in N,
and the per-cell minima against a plain loop."""
import numpy as np
import pytest

from oracle import dcalc as D


def _lattice(k, s, x0=1000, y0=2000):
    i, j = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    return np.stack([x0 + s * i.ravel(), y0 + s * j.ravel()], 1).astype(np.int32), i.ravel(), j.ravel()


def test_lattice_closed_forms():
    s = 7
    xy, i, j = _lattice(6, s)
    corner = ((i == 0) | (i == 5)) & ((j == 0) | (j == 5))
    edge = ((i == 0) | (i == 5) | (j == 0) | (j == 5)) & ~corner
    inner = ~(corner | edge)
    # N = 1: every point has a neighbour at one spacing
    assert np.all(D.nth_nn_dist2(xy, 1) == s * s)
    # N = 4: interior: four at s; edge: three at s, then the diagonal 2 s^2;
    # corner: two at s, one diagonal 2 s^2, then two at 2 s (4 s^2)
    d4 = D.nth_nn_dist2(xy, 4)
    assert np.all(d4[inner] == s * s)
    assert np.all(d4[edge] == 2 * s * s)
    assert np.all(d4[corner] == 4 * s * s)
    # N = 5: interior: the first diagonal; edge: the second diagonal; corner: 4 s^2
    d5 = D.nth_nn_dist2(xy, 5)
    assert np.all(d5[inner] == 2 * s * s)
    assert np.all(d5[edge] == 2 * s * s)
    assert np.all(d5[corner] == 4 * s * s)


def test_hand_example():
    xy = np.array([[0, 0], [3, 0], [0, 4], [10, 10]], dtype=np.int32)
    # from (0,0): 9, 16, 200; from (3,0): 9, 25, 149; from (0,4): 16, 25, 136;
    # from (10,10): 136, 149, 200
    assert D.nth_nn_dist2(xy, 1).tolist() == [9, 9, 16, 136]
    assert D.nth_nn_dist2(xy, 2).tolist() == [16, 25, 25, 149]
    assert D.nth_nn_dist2(xy, 3).tolist() == [200, 149, 136, 200]
    with pytest.raises(ValueError):
        D.nth_nn_dist2(xy, 4)


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_matches_kdtree(N):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(N)
    xy = np.unique(rng.integers(0, 1 << 16, size=(3000, 2)), axis=0).astype(np.int32)
    got = D.nth_nn_dist2(xy, N)
    dist, _ = spatial.cKDTree(xy.astype(np.float64)).query(xy.astype(np.float64), k=N + 1)
    exp = np.rint(dist[:, N] ** 2).astype(np.int64)  # exact: integer squares far below 2^52
    assert np.array_equal(got, exp)


def test_monotone_in_n_and_cells():
    rng = np.random.default_rng(3)
    xy = np.unique(rng.integers(0, 1 << 12, size=(800, 2)), axis=0).astype(np.int32)
    prev = None
    for N in range(1, 7):
        d = D.nth_nn_dist2(xy, N)
        if prev is not None:
            assert np.all(d >= prev)
        prev = d
    G, bits = 4, 12
    dist2, cmin, m = D.d_values(xy, 3, G, bits)
    for c in range(G * G):
        sel = [k for k in range(xy.shape[0]) if (int(xy[k, 1]) * G >> bits) * G + (int(xy[k, 0]) * G >> bits) == c]
        assert cmin[c] == (min(dist2[sel]) if sel else D.NONE)
    assert m == dist2.min()
    # a block's N-spread: its cell's diagonal over d
    assert D.n_spread(G, bits, 4) == pytest.approx(1024 * np.sqrt(2) / 2)


PLANTS = {
    "control": None,
    "n_off_by_one": ("np.partition(d2, N - 1, axis=1)[:, N - 1]", "np.partition(d2, N, axis=1)[:, N]"),
    "self_counted": ("d2[np.arange(A.shape[0]), np.arange(s, s + A.shape[0])] = NONE", "pass"),
    "dy_dropped": ("d2 = dx * dx + dy * dy", "d2 = dx * dx"),
    "cells_transposed": ("return cy * grid + cx", "return cx * grid + cy"),
    "cell_max": ("np.minimum.at(cmin, cell, dist2)", "cmin[:] = 0; np.maximum.at(cmin, cell, dist2)"),
}


def _planted(name):
    import types
    src = open(D.__file__).read()
    if PLANTS[name] is not None:
        old, new = PLANTS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    mod = types.ModuleType("dcalc_planted")
    exec(compile(src, "dcalc_planted", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", list(PLANTS))
def test_plant_is_caught(name, monkeypatch):
    """Each planted mistake fails at least one pin; the unmodified copy passes all."""
    pins = [test_lattice_closed_forms, test_hand_example, test_monotone_in_n_and_cells]
    monkeypatch.setitem(globals(), "D", _planted(name))
    failed = 0
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    if name == "control":
        assert failed == 0
    else:
        assert failed > 0, name
