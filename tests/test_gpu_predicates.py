"""Device predicates against the oracle's and against exact big-integer forms."""
import numpy as np
import pytest

import oracle
from tests import _pins

pytestmark = pytest.mark.gpu


def _run(xy, quads, use_filter=True):
    import torch
    from paper_2308_06484_gb300 import kdt
    dxy = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(quads, dtype=np.int32)).cuda()
    out = torch.empty((quads.shape[0], 4), dtype=torch.int32, device="cuda")
    kdt.eval_predicates(dxy, dq, out, use_filter)
    return out.cpu().numpy()


@pytest.mark.parametrize("span", [1 << 6, 1 << 16, 1 << 24, 1 << 28])
def test_random_quads_match_oracle(span):
    rng = np.random.default_rng(span)
    n = 4000
    xy = rng.integers(0, span, size=(n, 2)).astype(np.int32)
    q = np.stack([rng.choice(n, 4, replace=False) for _ in range(20000)]).astype(np.int32)
    out = _run(xy, q)
    for i in range(0, q.shape[0], 7):
        a, b, c, d = (int(v) for v in q[i])
        assert out[i, 0] == oracle.orient2d(xy, a, b, c)
        assert out[i, 1] == oracle.incircle_raw(xy, a, b, c, d)
        assert out[i, 3] == oracle.incircle_sos(xy, a, b, c, d)
    # the filter never contradicts the exact sign
    f = out[:, 2]
    assert np.all((f == 0) | (f == out[:, 1]))


def test_cocircular_lattice_sos():
    g = np.array([(x, y) for x in range(6) for y in range(6)], dtype=np.int32) * 64 + 1000
    rng = np.random.default_rng(5)
    perm = rng.permutation(len(g))
    xy = g[perm]
    q = np.stack([rng.choice(len(g), 4, replace=False) for _ in range(30000)]).astype(np.int32)
    out = _run(xy, q)
    ties = 0
    for i in range(q.shape[0]):
        a, b, c, d = (int(v) for v in q[i])
        if out[i, 1] == 0:
            ties += 1
            assert out[i, 3] == oracle.incircle_sos(xy, a, b, c, d)
    assert ties > 500


def test_near_degenerate_filter_is_safe():
    """Perturbed cocircular quadruples at full 2^28 scale: the FP32 filter must only
    answer when its sign is the exact one."""
    rng = np.random.default_rng(9)
    m = 200000
    R = rng.integers(1 << 20, 1 << 26, size=m)
    cx = rng.integers(1 << 26, (1 << 28) - (1 << 27), size=m)
    cy = rng.integers(1 << 26, (1 << 28) - (1 << 27), size=m)
    pts = []
    # Pythagorean-like points on a circle: (R,0), (0,R), (-R,0) plus a jittered 4th
    for k in range(m):
        j = rng.integers(-2, 3, size=2)
        pts += [(cx[k] + R[k], cy[k]), (cx[k], cy[k] + R[k]), (cx[k] - R[k], cy[k]),
                (cx[k] + j[0], cy[k] - R[k] + j[1])]
    xy = np.array(pts, dtype=np.int64)
    assert xy.min() >= 0 and xy.max() < (1 << 28)
    q = np.arange(4 * m, dtype=np.int32).reshape(m, 4)
    out = _run(xy.astype(np.int32), q)
    f = out[:, 2]
    assert np.all((f == 0) | (f == out[:, 1]))
    assert (f == 0).sum() > 0  # the filter does defer on near-ties
    for i in range(0, m, 997):
        a, b, c, d = (int(v) for v in q[i])
        assert out[i, 1] == _pins.sign(_pins.det4_lifted(xy[[a, b, c, d]]))


def test_exact_only_equals_filtered():
    rng = np.random.default_rng(3)
    xy = rng.integers(0, 1 << 24, size=(1000, 2)).astype(np.int32)
    q = np.stack([rng.choice(1000, 4, replace=False) for _ in range(5000)]).astype(np.int32)
    assert np.array_equal(_run(xy, q, True)[:, 3], _run(xy, q, False)[:, 3])
