"""d-calculation on the GPU (kdt_d_values) against the brute-force reference in
oracle/dcalc.py, exactly: every point's N-th nearest-neighbour squared distance, the
per-partition minima, mindistance, the running d over steps, and the block N-spread."""
import numpy as np
import pytest

from oracle import dcalc as D
from paper_2308_06484_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tri(**kw):
    from paper_2308_06484_gb300 import kdt
    return kdt.Triangulation(kdt.default_config(**kw))


def _check(t, xy, N, G, bits, device=False):
    import torch
    n = xy.shape[0]
    if device:
        dist2 = torch.empty(n, dtype=torch.int64, device="cuda")
        cmin = torch.empty(t.num_cells(), dtype=torch.int64, device="cuda")
    else:
        dist2 = np.empty(n, dtype=np.int64)
        cmin = np.empty(t.num_cells(), dtype=np.int64)
    info = t.d_values(N, dist2, cmin)
    if device:
        torch.cuda.synchronize()
        dist2, cmin = dist2.cpu().numpy(), cmin.cpu().numpy()
    e_dist, e_cmin, e_min = D.d_values(xy, N, G, bits)
    assert np.array_equal(dist2, e_dist), (N, np.nonzero(dist2 != e_dist)[0][:5])
    assert np.array_equal(cmin, e_cmin)
    assert info["min2"] == e_min
    assert info["cells"] == G * G
    return info


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
def test_c1_points(N):
    w = W.c1()
    t = _tri(grid=w.grid, domain_bits=w.bits)
    t.build(w.positions)
    info = _check(t, w.positions, N, w.grid, w.bits, device=(N % 2 == 0))
    assert info["d2"] == info["min2"]
    assert info["spread"] == pytest.approx(D.n_spread(w.grid, w.bits, info["d2"]), rel=1e-12)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_lattice_and_mixture(N):
    """Lattice patches: many equal distances (ties) and cocircular cells."""
    xy = W.mixture_lattice_points(20000, 24, 9)
    t = _tri(grid=16, domain_bits=24)
    t.build(xy)
    _check(t, xy, N, 16, 24)


def test_high_degree_points():
    """Points with 60-400 neighbours (a straight row beside sparse points)."""
    from tests.test_gpu_kinetic import _row_points
    xy, _ = _row_points(61)
    t = _tri(grid=16, domain_bits=22)
    t.build(xy)
    for N in (1, 2, 5):
        info = _check(t, xy, N, 16, 22)
    assert info["max_degree"] > 64


def test_running_d_over_steps():
    """d = min over the steps of mindistance(P_t); a new N or a new build starts again."""
    import torch
    w = W.c2(n=20000, grid=16, seed=12)
    t = _tri(grid=16, domain_bits=24)
    t.build(w.positions)
    run = None
    for s in range(4):
        info = t.d_values(2)
        e = int(D.nth_nn_dist2(w.positions, 2).min())
        run = e if run is None else min(run, e)
        assert info["min2"] == e and info["d2"] == run
        t.step(torch.from_numpy(w.next_moves()).cuda())
    info = t.d_values(1)  # another N: the minimum starts again
    assert info["d2"] == info["min2"] == int(D.nth_nn_dist2(w.positions, 1).min())
    t.build(w.positions)
    info = t.d_values(1)
    assert info["d2"] == info["min2"]


def test_batch_instances():
    """Each instance's points find their neighbours in their own instance."""
    from paper_2308_06484_gb300 import kdt
    rng = np.random.default_rng(5)
    sizes = [40, 300, 1200]
    parts = [np.unique(rng.integers(0, 1 << 20, size=(m, 2)), axis=0).astype(np.int32) for m in sizes]
    offs = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])]).astype(np.int64)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20))
    t.build_batch(parts)
    dist2 = np.empty(int(offs[-1]), dtype=np.int64)
    cmin = np.empty(t.num_cells(), dtype=np.int64)
    info = t.d_values(3, dist2, cmin)
    exp = np.concatenate([D.nth_nn_dist2(p, 3) for p in parts])
    assert np.array_equal(dist2, exp)
    assert info["min2"] == exp.min()
    assert info["spread"] == 0.0
    assert cmin.min() == exp.min() and cmin.shape[0] == info["cells"]


def test_errors():
    from paper_2308_06484_gb300 import kdt
    t = _tri(grid=4, domain_bits=16)
    with pytest.raises(kdt.KDTError):
        t.d_values(1)  # not built
    t.build(W.uniform_points(10, 16, 3))
    for N in (0, 17, 10):
        with pytest.raises(kdt.KDTError):
            t.d_values(N)
    assert t.d_values(9)["min2"] > 0
