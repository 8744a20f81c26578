"""The learned locate proposal on the GPU, against the CPU references in oracle/:
network outputs and gradients (FP32, BF16-rounded weights, rel. tol 1e-3), the Adam
step and its BF16 rounding, the training rows the kinetic kernel records (slot and
cavity exact, features to the last bit), and the triangulation with the proposal on
(bit-exact against the oracle)."""
import numpy as np
import pytest

import oracle
from oracle import mlp_ref as M
from oracle import trace_ref as TR
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same

pytestmark = pytest.mark.gpu


def _tri():
    from paper_2308_06484_gb300 import kdt
    return kdt.Triangulation(kdt.default_config(domain_bits=24))


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    theta = (M.init_params(seed) * scale + rng.normal(0, 0.02, M.N_PARAMS)).astype(np.float32)
    return M.bf16_round(theta), M.bf16_bits(theta)


def _batch(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, 32)).astype(np.float32)
    y = np.stack([rng.integers(0, 17, rows), rng.integers(1, 40, rows)], axis=1).astype(np.int32)
    return X, y


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("rows", [1, 37, 1000])
def test_forward_matches_reference(rows):
    import torch
    t = _tri()
    theta, bits = _params(1)
    X, _ = _batch(rows, 2)
    out = torch.empty((rows, 18), dtype=torch.float32, device="cuda")
    t.mlp_forward(_cuda(bits.view(np.int16)), _cuda(X), out)
    torch.cuda.synchronize()
    ref, _ = M.forward(theta, X)
    got = out.cpu().numpy()
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(got - ref) / scale) < 1e-5


@pytest.mark.parametrize("rows,use_index", [(33, False), (1000, False), (4099, True)])
def test_loss_and_gradient_match_reference(rows, use_index):
    """Gradient check against the CPU FP32 reference with the same BF16-rounded weights."""
    import torch
    t = _tri()
    theta, bits = _params(3, scale=0.8)
    X, y = _batch(rows, 4)
    lam = 0.25
    index = None
    sel = np.arange(rows)
    if use_index:
        sel = np.random.default_rng(5).permutation(rows)[: rows - 7]
        index = _cuda(sel.astype(np.int64))
    grad = torch.zeros(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    t.mlp_loss_grad(_cuda(bits.view(np.int16)), _cuda(X), _cuda(y), grad, loss, index=index, lam=lam)
    torch.cuda.synchronize()
    lref, gref = M.loss_and_grad(theta, X[sel], y[sel, 0], y[sel, 1], lam, np.float32)
    g = grad.cpu().numpy()
    assert abs(float(loss.item()) - float(lref)) <= 1e-3 * abs(float(lref))
    # every tensor within 1e-3 of its largest entry, every large entry within 1e-3 of itself
    o = 0
    for _, shape in M.SIZES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], gref[o:o + k]
        mx = float(np.max(np.abs(b)))
        assert np.max(np.abs(a - b)) <= 1e-3 * mx + 1e-12, shape
        big = np.abs(b) > 0.05 * mx
        assert np.all(np.abs(a[big] - b[big]) <= 1e-3 * np.abs(b[big])), shape
        o += k
    # the same call again gives the same bits (fixed summation order)
    g1 = grad.clone()
    t.mlp_loss_grad(_cuda(bits.view(np.int16)), _cuda(X), _cuda(y), grad, loss, index=index, lam=lam)
    torch.cuda.synchronize()
    assert torch.equal(g1, grad)


def test_adam_and_bf16_rounding_match_reference():
    import torch
    t = _tri()
    rng = np.random.default_rng(8)
    master = rng.standard_normal(M.N_PARAMS).astype(np.float32)
    m = np.zeros_like(master)
    v = np.zeros_like(master)
    dm, dmm, dv = _cuda(master.copy()), _cuda(m.copy()), _cuda(v.copy())
    bits = torch.zeros(M.N_PARAMS, dtype=torch.int16, device="cuda")
    for step in range(1, 4):
        g = rng.standard_normal(M.N_PARAMS).astype(np.float32)
        M.adam_step(master, g, m, v, step, 1e-2, 0.9, 0.99, 1e-7)
        t.mlp_adam(dm, _cuda(g), dmm, dv, step, 1e-2, 0.9, 0.99, 1e-7, bits)
    torch.cuda.synchronize()
    got = dm.cpu().numpy()
    assert np.allclose(got, master, rtol=1e-5, atol=1e-6)
    # BF16 rounding of the masters the GPU holds: round to nearest, ties to even
    assert np.array_equal(bits.cpu().numpy().view(np.uint16), M.bf16_bits(got))


def _single_moves(xy, count, seed, bits=16, span=(1, 40)):
    rng = np.random.default_rng(seed)
    cur = xy.copy()
    occ = set(map(tuple, cur.tolist()))
    for _ in range(count):
        p = int(rng.integers(0, cur.shape[0]))
        d = [(1, 0), (-1, 0), (0, 1), (0, -1)][int(rng.integers(0, 4))]
        s = int(rng.integers(span[0], span[1] + 1))
        q = (int(cur[p][0]) + d[0] * s, int(cur[p][1]) + d[1] * s)
        if not (0 <= q[0] < 1 << bits and 0 <= q[1] < 1 << bits) or q in occ:
            continue
        yield p, q, cur.copy()
        occ.discard(tuple(cur[p]))
        occ.add(q)
        cur[p] = q


def test_training_rows_match_oracle():
    """Every recorded row equals the CPU definition on the triangulation in force."""
    import torch
    from paper_2308_06484_gb300 import proposal
    xy = W.uniform_points(300, 12, 21)
    t = _tri()
    t.build(xy)
    tr = proposal.Trace(64)
    checked = slots = 0
    seen = set()
    for p, q, before in _single_moves(xy, 120, 22, bits=12):
        tr.attach(t)
        t.step(np.array([[p, q[0], q[1]]], dtype=np.int32))
        n = tr.detach(t)
        ref = TR.row(before, p, q)
        if n == 0:
            continue  # a hull point, or a move finished on the global path
        assert n == 1
        assert ref is not None, "a row for a hull point"
        f, s, c, _ = ref
        x, y = tr.view()
        assert (int(y[0, 0]), int(y[0, 1])) == (s, c), (p, q)
        assert np.array_equal(x[0].cpu().numpy().view(np.uint32), f.view(np.uint32)), (p, q)
        checked += 1
        seen.add(s)
    assert checked > 60
    assert len(seen) >= 3
    assert t.verify() == 0


def test_proposal_keeps_the_triangulation_exact():
    """Steps with the proposal on (a briefly trained network) equal the oracle."""
    import torch
    from paper_2308_06484_gb300 import kdt, proposal
    w = W.c2(n=20000, grid=8, seed=31)
    t = kdt.Triangulation(kdt.default_config(grid=8, domain_bits=24))
    t.build(w.positions)
    tr = proposal.Trace(20000)
    tr.attach(t)
    for _ in range(30):
        t.step(w.next_moves())
    tr.detach(t)
    x, y = tr.view()
    assert x.shape[0] > 1000
    tn = proposal.Trainer(t, seed=1)
    tn.fit(x, y, epochs=4, batch=512)
    acc, _ = tn.evaluate(x, y)
    t.set_proposal(tn.params)
    t.reset_stats()
    for s in range(10):
        t.step(w.next_moves())
        if s % 3 == 2:
            assert_same(t.export_triangles(), w.positions, "proposal step %d" % s)
    st = t.stats()
    assert st["proposal_moves"] > 0
    assert 0 < st["proposal_hits"] <= st["proposal_moves"]
    assert t.verify() == 0
    assert acc > 0.25
    t.set_proposal(None)
    t.step(w.next_moves())
    assert_same(t.export_triangles(), w.positions, "proposal off")
