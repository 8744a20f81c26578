"""Pins for the quad-tree partitioning reference (no GPU): a hand example with the
paper's threshold 2 (Section III, Fig. 2), the defining properties on random and
clustered sets (leaves tile the square, every leaf within the threshold unless at the
depth limit, every divided square above it), and the numbering order."""
import numpy as np

from oracle import quadtree as Q


def test_hand_example_threshold_two():
    # square [0, 8)^2 (extent 8); five points, threshold 2
    xy = np.array([[0, 0], [1, 1], [2, 2], [7, 7], [6, 1]], dtype=np.int32)
    sq, lay = Q.leaves(xy, 2)
    assert lay == (0, 0, 3, 3)
    # root (5 > 2) -> four 4x4 squares: (0,0) holds 3 points -> divided again into 2x2:
    # (0,0) 2 points [(0,0), (1,1)], (2,0) 0, (0,2) 0, (2,2) 1; then (4,0) 1, (0,4) 0, (4,4) 1
    assert sq == [(0, 0, 2), (2, 0, 2), (0, 2, 2), (2, 2, 2), (4, 0, 4), (0, 4, 4), (4, 4, 4)]
    assert Q.block_of(xy, sq, lay).tolist() == [0, 0, 3, 6, 4]
    # clamped positions (outside the square after a move)
    assert Q.block_of(np.array([[-5, -5], [100, 3]]), sq, lay).tolist() == [0, 4]


def _check_properties(xy, T):
    sq, (x0, y0, lg, D) = Q.leaves(xy, T)
    side = 1 << lg
    assert sum(s * s for _, _, s in sq) == side * side  # the leaves tile the square
    blk = Q.block_of(xy, sq, (x0, y0, lg, D))
    assert np.all(blk >= 0)
    counts = np.bincount(blk, minlength=len(sq))
    min_side = side >> D
    for (x, y, s), c in zip(sq, counts):
        assert c <= T or s == min_side
        # the parent square of a leaf held more than T points (it was divided)
        if s < side:
            px, py = x - (x - x0) % (2 * s), y - (y - y0) % (2 * s)
            inside = ((xy[:, 0] >= px) & (xy[:, 0] < px + 2 * s) & (xy[:, 1] >= py) & (xy[:, 1] < py + 2 * s))
            assert inside.sum() > T
    # depth-first order: a leaf's lower-left corner Morton code (relative to the
    # square, at the finest level) increases along the order
    def morton(x, y):
        fx, fy = (x - x0) // min_side, (y - y0) // min_side
        code = 0
        for b in range(D):
            code |= ((fx >> b) & 1) << (2 * b) | ((fy >> b) & 1) << (2 * b + 1)
        return code
    codes = [morton(x, y) for x, y, _ in sq]
    assert codes == sorted(codes)
    return sq


def test_properties_uniform_and_clustered():
    rng = np.random.default_rng(4)
    u = np.unique(rng.integers(0, 1 << 16, size=(3000, 2)), axis=0)
    _check_properties(u, 64)
    c = np.unique(np.clip(np.rint(rng.normal(30000, 300, size=(3000, 2))), 0, 65535).astype(np.int64), axis=0)
    sq = _check_properties(np.concatenate([c, u[:200]]), 32)
    assert len({s for _, _, s in sq}) > 3  # adaptive: squares of many sizes


def test_depth_limit():
    # 40 points on a 5x8 block of adjacent integers: the square (side 8) can only be
    # divided down to side 1, where a leaf holds one point
    xy = np.array([[x, y] for x in range(5) for y in range(8)], dtype=np.int32)
    sq, lay = Q.leaves(xy, 1)
    assert lay[2] == 3 and lay[3] == 3
    blk = Q.block_of(xy, sq, lay)
    assert np.bincount(blk).max() == 1


PLANTS = {
    "control": None,
    "threshold_off_by_one": ("if idx.size <= T or depth == D:", "if idx.size < T or depth == D:"),
    "children_order": ("        for cy in (0, 1):\n            for cx in (0, 1):",
                       "        for cx in (0, 1):\n            for cy in (0, 1):"),
    "side_too_small": ("while (1 << lg) < ext:", "while (2 << lg) < ext:"),
    "no_clamp": ("qx = np.clip(Q[:, 0], x0, x0 + side - 1)", "qx = Q[:, 0]"),
    "no_depth_limit": ("return x0, y0, lg, min(MAX_DEPTH, lg)", "return x0, y0, lg, MAX_DEPTH"),
}


def test_plants_are_caught():
    import types
    import pytest
    src0 = open(Q.__file__).read()
    for name, plant in PLANTS.items():
        src = src0
        if plant is not None:
            assert src.count(plant[0]) == 1, name
            src = src.replace(plant[0], plant[1])
        mod = types.ModuleType("qt_planted")
        exec(compile(src, "qt_planted", "exec"), mod.__dict__)
        failed = 0
        for pin in (test_hand_example_threshold_two, test_properties_uniform_and_clustered, test_depth_limit):
            g = pin.__globals__
            old = g["Q"]
            g["Q"] = mod
            try:
                pin()
            except Exception:
                failed += 1
            finally:
                g["Q"] = old
        assert (failed == 0) if plant is None else (failed > 0), name


def test_redivision_in_a_given_square():
    """A division repeated with the build's layout clamps positions into its square and
    equals a fresh division when every position is inside it."""
    import numpy as np
    from oracle import quadtree as Q
    rng = np.random.default_rng(5)
    xy = rng.integers(100, 900, size=(400, 2))
    sq, lay = Q.leaves(xy, 8)
    assert Q.leaves(xy, 8, lay=lay)[0] == sq
    moved = xy.copy()
    moved[:40] = [[-50, 5000]] * 40  # outside: clamped to the top-left corner's leaf
    sq2, _ = Q.leaves(moved, 8, lay=lay)
    cl = np.stack([np.clip(moved[:, 0], lay[0], lay[0] + (1 << lay[2]) - 1),
                   np.clip(moved[:, 1], lay[1], lay[1] + (1 << lay[2]) - 1)], axis=1)
    assert sq2 == Q.leaves(cl, 8, lay=lay)[0]
    assert sq2 != sq  # 40 points piled into one corner divide it further
    blocks = Q.block_of(moved, sq2, lay)
    assert (blocks >= 0).all()
    counts = np.bincount(blocks, minlength=len(sq2))
    side0 = 1 << lay[2]
    assert sum(s * s for _, _, s in sq2) == side0 * side0  # the leaves tile the square
    for (x, y, side), c in zip(sq2, counts):
        assert c <= 8 or side == side0 >> lay[3]  # above the threshold only at the floor
