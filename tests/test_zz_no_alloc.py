"""The allocation-free export (kdt_export_triangles_noalloc) against the regular
export, through the C ABI.

Callers that cannot let the library call cudaMalloc (a device whose memory budget an
application already reserved for its own pool, a per-step output loop that must not
take the allocation path) use this entry point; its scratch is a fixed file-scope
device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2308_06484_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _export_noalloc(t, rows):
    import torch
    out = torch.full((rows, 3), -7, dtype=torch.int32, device="cuda")
    nt = t.export_triangles_noalloc(out)
    return out[:nt].cpu().numpy(), nt


def test_noalloc_matches_export_two_calls_in_a_row():
    from paper_2308_06484_gb300 import kdt
    import torch
    w = W.c2(n=200_000, grid=32)
    t = kdt.Triangulation(kdt.default_config(grid=w.grid, domain_bits=w.bits))
    t.build(w.positions)
    ref = t.export_triangles()
    for _ in range(2):  # the shared scratch keeps the last call's contents
        before = t.stats()["kernel_launches"]
        got, nt = _export_noalloc(t, ref.shape[0] + 5)
        # count, three scan passes, place, segment sort
        assert t.stats()["kernel_launches"] - before == 6
        assert nt == ref.shape[0]
        assert np.array_equal(got, ref)
    # after a time step the triangulation changes; the next call must follow it
    t.step(torch.from_numpy(w.next_moves()).cuda())
    ref2 = t.export_triangles()
    got, nt = _export_noalloc(t, ref2.shape[0])
    assert np.array_equal(got, ref2)


def test_noalloc_smaller_after_larger_and_errors():
    from paper_2308_06484_gb300 import kdt
    import torch
    big = kdt.Triangulation(kdt.default_config(domain_bits=24))
    big.build(W.uniform_points(100_000, 24, 3))
    _export_noalloc(big, 2 * 100_000)
    small = kdt.Triangulation(kdt.default_config(domain_bits=16))
    w = W.c1()
    small.build(w.positions)
    ref = small.export_triangles()
    got, nt = _export_noalloc(small, ref.shape[0])
    assert np.array_equal(got, ref)
    # too small an output buffer: the row count is still reported
    out = torch.empty((10, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(kdt.KDTError) as e:
        small.export_triangles_noalloc(out)
    assert e.value.name == "KDT_ERR_CAPACITY"
    # host output is rejected (it would need a staging buffer)
    with pytest.raises(kdt.KDTError) as e:
        small.export_triangles_noalloc(np.empty((ref.shape[0], 3), dtype=np.int32))
    assert e.value.name == "KDT_ERR_ARG"
    # beyond the documented maximum number of points
    n = (1 << 20) + 1
    huge = kdt.Triangulation(kdt.default_config(domain_bits=24))
    huge.build(W.uniform_points(n, 24, 4))
    out = torch.empty((2 * n, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(kdt.KDTError) as e:
        huge.export_triangles_noalloc(out)
    assert e.value.name == "KDT_ERR_TOO_LARGE"
