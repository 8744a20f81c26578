"""Batched instances (kdt_build_batch / kdt_step_batch, one launch per step for all
instances) against the oracle, instance by instance, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same

pytestmark = pytest.mark.gpu


def _batch(n_inst, lo, hi, seed):
    sizes = W.c4_sizes(n_inst, seed, lo, hi)
    ws = []
    for i, n_i in enumerate(sizes):
        xy = W.uniform_points(int(n_i), 20, seed * 100003 + i)
        ws.append(W.KineticWorkload(xy, grid=W.c4_grid(int(n_i)), bits=20, moves_per_cell=(1, 4),
                                    dist=(1, 8), seed=seed * 7919 + i, name="b%d" % i))
    return ws


def _step_moves(ws):
    mv = [w.next_moves() for w in ws]
    offs = np.zeros(len(mv) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([m.shape[0] for m in mv])
    return np.ascontiguousarray(np.concatenate(mv)), offs


def _check_all(t, ws, what):
    for i, w in enumerate(ws):
        assert_same(t.export_triangles_inst(i), w.positions, "%s instance %d" % (what, i))


@pytest.mark.parametrize("autotune", [0, 1])
def test_batch_steps_match_oracle(autotune):
    import torch
    from paper_2308_06484_gb300 import kdt
    ws = _batch(24, 300, 6000, seed=41 + autotune)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20, autotune=autotune))
    t.build_batch([w.positions for w in ws])
    assert t.n_instances == 24
    _check_all(t, ws, "build")
    for s in range(20 if autotune else 6):
        mv, offs = _step_moves(ws)
        t.step_batch(torch.from_numpy(mv).cuda() if s % 2 else mv, offs)
        if s % 3 == 2 or s == 5:
            _check_all(t, ws, "step %d" % s)
    _check_all(t, ws, "final")
    assert t.verify() == 0
    st = t.stats()
    assert st["fallbacks"] == 0
    if autotune:
        assert st["tuned_points_per_partition"] in (128, 256, 512)
        assert st["tuned_warps_per_partition"] in (1, 2, 4)


def test_batch_global_export_and_points():
    from paper_2308_06484_gb300 import kdt
    ws = _batch(5, 50, 400, seed=7)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20))
    t.build_batch([w.positions for w in ws])
    allt = t.export_triangles()
    offs = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    parts = [t.export_triangles_inst(i) + offs[i] for i in range(len(ws))]
    assert np.array_equal(allt, np.concatenate(parts))
    assert np.array_equal(t.export_points(), np.concatenate([w.positions for w in ws]))


def test_batch_errors():
    from paper_2308_06484_gb300 import kdt
    ws = _batch(3, 50, 100, seed=9)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20))
    t.build_batch([w.positions for w in ws])
    before = [t.export_triangles_inst(i).copy() for i in range(3)]
    # a local id beyond its instance
    mv = np.array([[ws[1].n, 5, 5]], dtype=np.int32)
    with pytest.raises(kdt.KDTError) as e:
        t.step_batch(mv, [0, 0, 1, 1])
    assert e.value.name == "KDT_ERR_ARG"
    # the single-instance step is refused on a batched handle
    with pytest.raises(kdt.KDTError) as e:
        t.step(mv)
    assert e.value.name == "KDT_ERR_STATE"
    for i in range(3):
        assert np.array_equal(t.export_triangles_inst(i), before[i])
    with pytest.raises(kdt.KDTError):
        t.build_batch([w.positions[:2] for w in ws])  # an instance with 2 points


def test_batch_full_size_sampled():
    """The 512-instance workload at full size (2.2e7 points): after the build and two
    steps every triangle belongs to its own instance (kdt_verify) and sampled
    instances equal the oracle."""
    from paper_2308_06484_gb300 import kdt
    ws = W.c4()
    t = kdt.Triangulation(kdt.default_config(domain_bits=20))
    t.build_batch([w.positions for w in ws])
    sample = list(range(0, 512, 32)) + [1, 511]
    assert t.verify() == 0
    for i in sample:
        assert_same(t.export_triangles_inst(i), ws[i].positions, "build instance %d" % i)
    for s in range(2):
        mv, offs = _step_moves(ws)
        t.step_batch(mv, offs)
    assert t.verify() == 0
    for i in sample:
        assert_same(t.export_triangles_inst(i), ws[i].positions, "step instance %d" % i)
    assert t.stats()["fallbacks"] == 0


def test_batched_build_equals_one_instance_at_a_time():
    """kdt_config.batch_build: every instance built in one set of launches gives the same
    triangulations as building them one after another, and as the oracle; including
    3-point instances, an instance whose first points are collinear, a lattice and
    repeated rebuilds after steps."""
    import torch
    from paper_2308_06484_gb300 import kdt
    ws = _batch(20, 3, 5000, seed=71)
    rng = np.random.default_rng(72)
    line = np.stack([np.arange(40) * 3 + 5, np.full(40, 77)], axis=1)
    line = np.concatenate([line, [[60, 500], [61, 9]]]).astype(np.int32)  # collinear first, then two off the line
    g = np.arange(12)
    lat = (np.stack(np.meshgrid(g, g), -1).reshape(-1, 2) * 64 + 1000).astype(np.int32)
    xys = [w.positions for w in ws] + [line, lat, np.array([[1, 1], [9, 2], [4, 8]], dtype=np.int32)]
    ts = {}
    for bb in (0, 1):
        t = kdt.Triangulation(kdt.default_config(domain_bits=20, batch_build=bb))
        t.build_batch(xys)
        ts[bb] = t
    for i, xy in enumerate(xys):
        a = ts[1].export_triangles_inst(i)
        assert np.array_equal(a, ts[0].export_triangles_inst(i)), i
        assert_same(a, xy, "batched build instance %d" % i)
    assert ts[1].verify() == 0
    for s in range(3):
        mv, offs = _step_moves(ws)
        offs = np.concatenate([offs, [offs[-1]] * 3])
        ts[1].step_batch(torch.from_numpy(mv).cuda(), offs)
        ts[1].rebuild()
    for i, w in enumerate(ws):
        assert_same(ts[1].export_triangles_inst(i), w.positions, "rebuilt instance %d" % i)
    assert ts[1].verify() == 0
    for t in ts.values():
        t.close()
