"""Shared helpers of the GPU parity tests (compare the CUDA path with the oracle)."""
import numpy as np

import oracle


def assert_same(got, xy, what=""):
    exp = oracle.delaunay(xy)
    if got.shape != exp.shape or not np.array_equal(got, exp):
        g = set(map(tuple, got.tolist()))
        e = set(map(tuple, exp.tolist()))
        raise AssertionError("%s: GPU %d rows vs oracle %d rows; %d missing, %d extra; first missing %s"
                             % (what, got.shape[0], exp.shape[0], len(e - g), len(g - e),
                                sorted(e - g)[:3]))


def run_kinetic(tri, w, steps, every=1, check_points=True):
    """Apply `steps` generated steps; compare with the oracle every `every` steps."""
    import torch
    for s in range(steps):
        mv = w.next_moves()
        tri.step(torch.from_numpy(mv).cuda())
        if (s + 1) % every == 0 or s == steps - 1:
            if check_points:
                assert np.array_equal(tri.export_points(), w.positions)
            assert_same(tri.export_triangles(), w.positions, "%s step %d" % (w.name, s + 1))
