"""d-calculation reference — TEST INFRASTRUCTURE ONLY (only the tests, the smoke run
and bench.py's CPU legs may import it; it shares no code with the CUDA path).

Section III ("Notation and definitions") fixes a constant N and, for every point p,
dist_p = the distance from p to its N-th nearest neighbour; mindistance(P) is the
minimum of dist_p over the points and d = min over the time steps of
mindistance(P_t).  Section IV ("d-calculation") computes the minimum per block first
and then over all blocks.  Section III also defines the N-spread of a block,
Delta_N(P_i) = diam(P_i) / mindistance(P), with the block's diameter taken from the
partition (the grid cell, whose diagonal every block shares here).

Everything is exact integer arithmetic on squared distances (coordinates below 2^28,
so a squared distance is below 2^57): the N-th smallest squared distance from p to
the other points, by brute force over all pairs (the definition written out).  Ties
do not matter: the N-th smallest value is unique even when the N-th neighbour is not.
"""
import numpy as np

NONE = np.iinfo(np.int64).max  # an empty cell's minimum


def nth_nn_dist2(xy, N, chunk=2048):
    """Squared distance from every point to its N-th nearest other point (N >= 1)."""
    P = np.asarray(xy, dtype=np.int64)
    n = P.shape[0]
    if not 1 <= N < n:
        raise ValueError("need 1 <= N < n")
    out = np.empty(n, dtype=np.int64)
    for s in range(0, n, chunk):
        A = P[s:s + chunk]
        dx = A[:, None, 0] - P[None, :, 0]
        dy = A[:, None, 1] - P[None, :, 1]
        d2 = dx * dx + dy * dy
        d2[np.arange(A.shape[0]), np.arange(s, s + A.shape[0])] = NONE  # not its own neighbour
        out[s:s + chunk] = np.partition(d2, N - 1, axis=1)[:, N - 1]
    return out


def cells_of(xy, grid, bits):
    """Partition (grid cell) of each point: (x * G >> bits, y * G >> bits), row-major."""
    P = np.asarray(xy, dtype=np.int64)
    cx = (P[:, 0] * grid) >> bits
    cy = (P[:, 1] * grid) >> bits
    return cy * grid + cx


def d_values(xy, N, grid, bits):
    """(dist2 per point, min dist2 per cell (NONE when empty), mindistance(P)^2)."""
    dist2 = nth_nn_dist2(xy, N)
    cell = cells_of(xy, grid, bits)
    cmin = np.full(grid * grid, NONE, dtype=np.int64)
    np.minimum.at(cmin, cell, dist2)
    return dist2, cmin, int(dist2.min())


def n_spread(grid, bits, d2):
    """Delta_N of a block: its cell's diagonal over d (d2 = d squared)."""
    side = float(1 << bits) / grid
    return side * np.sqrt(2.0) / np.sqrt(float(d2))
