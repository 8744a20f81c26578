"""Quad-tree partitioning reference — TEST INFRASTRUCTURE ONLY (only the tests may
import it; it shares no code with the CUDA path).

Section III ("Data structure"): take the smallest square covering all points and a
threshold T; divide the square into four equal squares, and each of those again,
until every square holds at most T points.  Readings where the paper is silent:

- the square's lower-left corner is the points' minimum x and minimum y, and its side
  S is the smallest power of two >= the larger extent (max - min + 1), so every
  division falls on integer coordinates;
- division stops at squares of side S / 2^D (D = min(11, log2 S)): a square that small
  is a leaf even above the threshold;
- leaves are numbered depth-first, the four children of a square in the order
  (low x, low y), (high x, low y), (low x, high y), (high x, high y);
- a point's block is the leaf holding its position; a position outside the square
  (a point that moved after the division) belongs to the leaf it is clamped to.
"""
import numpy as np

MAX_DEPTH = 11


def layout(xy):
    """(x0, y0, log2 S, D) of the covering square and the division depth limit."""
    P = np.asarray(xy, dtype=np.int64)
    x0, y0 = int(P[:, 0].min()), int(P[:, 1].min())
    ext = max(int(P[:, 0].max()) - x0, int(P[:, 1].max()) - y0) + 1
    lg = 0
    while (1 << lg) < ext:
        lg += 1
    return x0, y0, lg, min(MAX_DEPTH, lg)


def leaves(xy, T, lay=None):
    """Leaf squares as (x, y, side) in their depth-first order (the block ids).  With
    `lay` (a layout from an earlier division) the division is made again inside that
    square, positions outside it clamped into it (a division repeated during the time
    loop keeps the square of the build)."""
    P = np.asarray(xy, dtype=np.int64)
    if lay is None:
        x0, y0, lg, D = layout(P)
    else:
        x0, y0, lg, D = lay
        P = np.stack([np.clip(P[:, 0], x0, x0 + (1 << lg) - 1), np.clip(P[:, 1], y0, y0 + (1 << lg) - 1)], axis=1)
    out = []

    def divide(x, y, side, idx, depth):
        if idx.size <= T or depth == D:
            out.append((x, y, side))
            return
        h = side // 2
        px, py = P[idx, 0], P[idx, 1]
        for cy in (0, 1):
            for cx in (0, 1):
                lo_x, lo_y = x + cx * h, y + cy * h
                sel = idx[(px >= lo_x) & (px < lo_x + h) & (py >= lo_y) & (py < lo_y + h)]
                divide(lo_x, lo_y, h, sel, depth + 1)

    divide(x0, y0, 1 << lg, np.arange(P.shape[0]), 0)
    return out, (x0, y0, lg, D)


def block_of(pos, sq, lay):
    """Leaf (block id) of each position in `pos` for the leaves `sq` of layout `lay`."""
    x0, y0, lg, _ = lay
    side = 1 << lg
    Q = np.asarray(pos, dtype=np.int64)
    qx = np.clip(Q[:, 0], x0, x0 + side - 1)
    qy = np.clip(Q[:, 1], y0, y0 + side - 1)
    out = np.full(Q.shape[0], -1, dtype=np.int64)
    for i, (x, y, s) in enumerate(sq):
        out[(qx >= x) & (qx < x + s) & (qy >= y) & (qy < y + s)] = i
    return out
