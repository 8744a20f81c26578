"""GPU full construction (kdt_build / kdt_rebuild) against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same

pytestmark = pytest.mark.gpu


def _tri(**kw):
    from paper_2308_06484_gb300 import kdt
    return kdt.Triangulation(kdt.default_config(**kw))


def _build_check(xy, **kw):
    t = _tri(**kw)
    t.build(np.ascontiguousarray(xy, dtype=np.int32))
    assert_same(t.export_triangles(), xy, "build n=%d" % len(xy))
    assert t.verify() == 0
    return t


@pytest.mark.parametrize("n", [3, 4, 5, 7, 10, 33, 100, 1000, 4099, 50000])
def test_uniform(n):
    xy = W.uniform_points(n, 16 if n < 5000 else 24, seed=n)
    _build_check(xy)


def test_c1_points_host_and_device_input():
    import torch
    w = W.c1()
    t = _build_check(w.positions)
    t2 = _tri()
    t2.build(torch.from_numpy(w.positions).cuda())
    assert np.array_equal(t2.export_triangles(), t.export_triangles())


@pytest.mark.parametrize("side", [3, 8, 40])
def test_lattice(side):
    g = np.array([(x, y) for x in range(side) for y in range(side)], dtype=np.int32) * 5 + 7
    rng = np.random.default_rng(side)
    _build_check(g[rng.permutation(len(g))])


def test_mixture_lattice():
    _build_check(W.mixture_lattice_points(60000, 24, 11))


def test_collinear_hull_and_lines():
    pts = [(x, 0) for x in range(0, 400, 4)] + [(0, y) for y in range(4, 400, 4)]
    pts += [(x, 400 - x) for x in range(4, 400, 4)]
    rng = np.random.default_rng(2)
    pts += [tuple(p) for p in rng.integers(1, 200, size=(50, 2))]
    xy = np.unique(np.array(pts, dtype=np.int32), axis=0)
    _build_check(xy[rng.permutation(len(xy))])


def test_one_line_plus_one():
    xy = np.array([(x * 3, 5) for x in range(200)] + [(7, 900)], dtype=np.int32)
    _build_check(xy)


def test_rebuild_is_identical():
    xy = W.uniform_points(20000, 20, seed=4)
    t = _build_check(xy)
    a = t.export_triangles()
    t.rebuild()
    assert np.array_equal(t.export_triangles(), a)


def test_errors():
    from paper_2308_06484_gb300 import kdt
    t = _tri()
    with pytest.raises(kdt.KDTError) as e:
        t.build(np.array([[0, 0], [1, 1], [2, 2], [5, 5]], dtype=np.int32))
    assert e.value.name == "KDT_ERR_DEGENERATE"
    with pytest.raises(kdt.KDTError) as e:
        t.build(np.array([[0, 0], [1, 0], [0, 1], [1, 0]], dtype=np.int32))
    assert e.value.name == "KDT_ERR_DUPLICATE"
    with pytest.raises(kdt.KDTError) as e:
        t.build(np.array([[0, 0], [1, 0], [0, 1 << 28]], dtype=np.int32))
    assert e.value.name == "KDT_ERR_RANGE"
    with pytest.raises(kdt.KDTError) as e:
        t.build(np.array([[0, 0], [1, 0]], dtype=np.int32))
    assert e.value.name == "KDT_ERR_DEGENERATE"
    with pytest.raises(kdt.KDTError) as e:
        t.step(np.zeros((1, 3), dtype=np.int32))
    assert e.value.name == "KDT_ERR_STATE"
    # an invalid build leaves no triangulation behind; a valid one works afterwards
    t.build(W.uniform_points(100, 16, 1))
    assert t.verify() == 0


def test_export_capacity():
    from paper_2308_06484_gb300 import kdt
    xy = W.uniform_points(500, 16, 8)
    t = _build_check(xy)
    small = np.empty((10, 3), dtype=np.int32)
    with pytest.raises(kdt.KDTError) as e:
        t.export_triangles(small)
    assert e.value.name == "KDT_ERR_CAPACITY"
