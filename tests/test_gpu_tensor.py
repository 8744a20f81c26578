"""The learned proposal's network on the tensor cores (tcgen05): kdt_mlp_forward_tc
against the oracle's network (oracle/mlp_ref.py, evaluated in FP64) within the error
bound the split-BF16 arithmetic gives, and the step planner's tensor-core form
(kdt_config.plan = 2 | 4) keeping the triangulation bit-exact with the oracle, one
instance and a batch, with a hit rate equal to the CUDA-core planner's up to near-ties.

Error bound.  Every activation x enters a layer as hi + lo (two BF16 values) with
|x - hi - lo| <= 2^-16 |x|; the weights are BF16 already, so each product is exact and
the tensor core's FP32 accumulation of the 2K products adds at most 2K * 2^-23 of their
magnitude sum (2^-16 for K = 64, even with truncating adds); with the bias, one layer's
error is below eps = 2^-15 of S = |W| s_in + |b|, s_in the magnitude bound of its input.
ReLU is 1-Lipschitz, so the error after three layers is below 3 eps S3, with
S1 = |W1||x| + |b1|, S2 = |W2| S1 + |b2|, S3 = |W3| S2 + |b3| (row by row)."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same
from tests.test_gpu_batch import _batch, _check_all, _step_moves
from tests.test_gpu_plan import _steps_ms, _trained
from tests.test_gpu_proposal import _cuda, _params

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -15


def _magnitude(theta, X):
    """S3 of every output (rows x 18)."""
    W1, b1, W2, b2, W3, b3 = [np.abs(np.asarray(a, dtype=np.float64)) for a in M.unpack(theta)]
    S1 = np.abs(np.asarray(X, dtype=np.float64)) @ W1.T + b1
    S2 = S1 @ W2.T + b2
    return S2 @ W3.T + b3


def _handle():
    from paper_2308_06484_gb300 import kdt
    return kdt.Triangulation(kdt.default_config(domain_bits=24))


@pytest.mark.parametrize("rows,scale", [(1, 1.0), (127, 1.0), (128, 1.0), (129, 1.0), (1000, 1.0),
                                        (70001, 1.0), (4099, 300.0)])
def test_forward_tc_within_bound(rows, scale):
    """Ragged tails (1, 127, 129 rows), whole tiles, several tiles per CTA (70001 rows
    over at most three CTAs per SM), and inputs far from unit scale."""
    import torch
    t = _handle()
    theta, bits = _params(3)
    rng = np.random.default_rng(rows)
    X = (rng.standard_normal((rows, 32)) * scale).astype(np.float32)
    out = torch.full((rows, 18), float("nan"), dtype=torch.float32, device="cuda")
    t.mlp_forward_tc(_cuda(bits.view(np.int16)), _cuda(X), out)
    got = out.cpu().numpy().astype(np.float64)
    ref, _ = M.forward(theta, X, np.float64)
    S3 = _magnitude(theta, X)
    bound = 3.0 * EPS * S3
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), (err.max(), bound[err > bound][:4])
    # the lo parts are used: BF16 activations alone leave errors of about 2^-14.5 of S3
    # (tests/test_split_precision.py); with them the kernel measured 2^-24 on a GB300
    assert np.max(err / S3) < 2.0 ** -19
    # the guesses equal the FP32 CUDA-core evaluation's wherever the two largest slot
    # logits are farther apart than twice the bound
    o32 = torch.empty((rows, 18), dtype=torch.float32, device="cuda")
    t.mlp_forward(_cuda(bits.view(np.int16)), _cuda(X), o32)
    o32 = o32.cpu().numpy().astype(np.float64)
    srt = np.sort(ref[:, :17], axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * bound[:, :17].max(axis=1)
    assert np.array_equal(np.argmax(got[clear, :17], axis=1), np.argmax(o32[clear, :17], axis=1))
    assert clear.mean() > 0.5  # the comparison is not vacuous
    assert t.stats()["tensor_timeouts"] == 0


def test_forward_tc_edge_arguments():
    import ctypes
    import torch
    t = _handle()
    _, bits = _params(4)
    w = _cuda(bits.view(np.int16))
    empty = torch.empty((0, 32), dtype=torch.float32, device="cuda")
    t.mlp_forward_tc(w, empty, torch.empty((0, 18), dtype=torch.float32, device="cuda"))  # no-op
    # a host input, and a misaligned parameter pointer, are rejected before any launch
    out = torch.zeros((4, 18), dtype=torch.float32, device="cuda")
    xh = np.zeros((4, 32), dtype=np.float32)
    vp = ctypes.c_void_p
    assert t.L.kdt_mlp_forward_tc(t.h, vp(w.data_ptr()), vp(xh.ctypes.data), 4, vp(out.data_ptr())) == -1
    xd = _cuda(xh)
    assert t.L.kdt_mlp_forward_tc(t.h, vp(w.data_ptr() + 2), vp(xd.data_ptr()), 4, vp(out.data_ptr())) == -1
    assert t.stats()["kernel_launches"] == 0


def test_planner_on_tensor_cores_keeps_the_triangulation():
    """The same steps with the network evaluated by the planner on the CUDA cores
    (plan = 2) and on the tensor cores (plan = 2 | 4, and with the planned order, 7):
    the oracle's triangulation after every step, and about the same hit rate."""
    import torch
    from paper_2308_06484_gb300 import kdt
    tn, holder, _ = _trained(seed=71)
    w = W.c2(n=120000, grid=32, seed=72)
    xy0 = np.array(w.positions)
    moves, finals = [], []
    for _ in range(8):
        moves.append(w.next_moves())
        finals.append(np.array(w.positions))
    res = {}
    for plan in (2, 6, 7):
        t = kdt.Triangulation(kdt.default_config(grid=32, domain_bits=24, plan=plan))
        t.build(xy0)
        t.set_proposal(tn.params)
        for s, mv in enumerate(moves):
            t.step(torch.from_numpy(mv).cuda())
            if s in (0, 3, 7):
                assert_same(t.export_triangles(), finals[s], "plan %d step %d" % (plan, s))
        st = t.stats()
        assert st["fallbacks"] == 0 and st["tensor_timeouts"] == 0
        assert t.verify() == 0
        res[plan] = st["proposal_hits"] / max(1, st["proposal_moves"])
        t.close()
    print("hit rates: CUDA cores %.4f, tensor cores %.4f, tensor cores + order %.4f" % (res[2], res[6], res[7]))
    assert res[6] > 0.3
    assert abs(res[6] - res[2]) < 0.01
    holder.close()


def test_batched_planner_on_tensor_cores_matches_oracle():
    import torch
    from paper_2308_06484_gb300 import kdt
    tn, holder, _ = _trained(seed=73)
    ws = _batch(12, 400, 6000, seed=74)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20, plan=6))
    t.build_batch([w.positions for w in ws])
    t.set_proposal(tn.params)
    for s in range(5):
        mv, offs = _step_moves(ws)
        t.step_batch(torch.from_numpy(mv).cuda(), offs)
        if s % 2 == 0:
            _check_all(t, ws, "tensor planner batch step %d" % s)
    st = t.stats()
    assert st["proposal_moves"] > 0 and st["proposal_hits"] > 0
    assert st["fallbacks"] == 0 and st["tensor_timeouts"] == 0
    assert t.verify() == 0
    holder.close()


def test_tensor_planner_time():
    """Steps of the 1e6-point workload with the planner's network on the CUDA cores and
    on the tensor cores (printed; the benchmark reports them at full size)."""
    import torch
    from paper_2308_06484_gb300 import kdt
    tn, holder, _ = _trained(seed=75)
    w = W.c2(n=1000000, grid=64, seed=76)
    xy0 = np.array(w.positions)
    moves = [torch.from_numpy(w.next_moves()).cuda() for _ in range(22)]
    ms = {}
    for plan in (0, 2, 6):
        t = kdt.Triangulation(kdt.default_config(grid=64, domain_bits=24, plan=plan))
        t.build(xy0)
        if plan:
            t.set_proposal(tn.params)
        ms[plan] = _steps_ms(t, moves) / 20
        assert_same(t.export_triangles(), w.positions, "plan %d" % plan)
        t.close()
    print("ms per step: plain %.4f, planner network on CUDA cores %.4f, on tensor cores %.4f"
          % (ms[0], ms[2], ms[6]))
    holder.close()


def _grad_check(g, gref):
    """The tolerance of the CUDA-core gradient test: every tensor within 1e-3 of its
    largest entry, every entry above 5 % of it within 1e-3 of itself."""
    o = 0
    for name, shape in M.SIZES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], gref[o:o + k]
        mx = float(np.max(np.abs(b)))
        assert np.max(np.abs(a - b)) <= 1e-3 * mx + 1e-12, name
        big = np.abs(b) > 0.05 * mx
        assert np.all(np.abs(a[big] - b[big]) <= 1e-3 * np.abs(b[big])), name
        o += k


@pytest.mark.parametrize("rows,use_index", [(1, False), (33, False), (128, False), (1000, False), (4099, True),
                                            (38989, False)])
def test_loss_grad_tc_matches_reference(rows, use_index):
    """One row, a ragged tile, one whole tile, several tiles, an index list, and more
    tiles than SMs (several tiles accumulated in TMEM by each CTA)."""
    import torch
    from tests.test_gpu_proposal import _batch as _xy
    t = _handle()
    theta, bits = _params(3, scale=0.8)
    X, y = _xy(rows, 4)
    lam = 0.25
    index, sel = None, np.arange(rows)
    if use_index:
        sel = np.random.default_rng(5).permutation(rows)[: rows - 7]
        index = _cuda(sel.astype(np.int64))
    grad = torch.zeros(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    args = (_cuda(bits.view(np.int16)), _cuda(X), _cuda(y), grad, loss)
    t.mlp_loss_grad(*args, index=index, lam=lam, tensor_cores=True)
    lref, gref = M.loss_and_grad(theta, X[sel], y[sel, 0], y[sel, 1], lam, np.float32)
    assert abs(float(loss.item()) - float(lref)) <= 1e-3 * abs(float(lref))
    _grad_check(grad.cpu().numpy(), gref)
    g1 = grad.clone()
    t.mlp_loss_grad(*args, index=index, lam=lam, tensor_cores=True)
    torch.cuda.synchronize()
    assert torch.equal(g1, grad)  # fixed summation order
    assert t.stats()["tensor_timeouts"] == 0


def test_training_on_tensor_cores():
    """The same training run with the gradient on the CUDA cores and on the tensor cores:
    about the same final loss and accuracy; the gradient kernels' times printed."""
    import torch
    from paper_2308_06484_gb300 import kdt, proposal
    x, y = proposal.collect_traces([(W.c2(n=100000, grid=32, seed=77), 25)], cap=200000)
    res = {}
    for tc in (False, True):
        holder = kdt.Triangulation(kdt.default_config())
        tn = proposal.Trainer(holder, seed=0, tensor_cores=tc)
        last = tn.fit(x, y, epochs=3, batch=4096, seed=0)
        acc, mae = tn.evaluate(x, y)
        grad = torch.zeros(M.N_PARAMS, dtype=torch.float32, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            holder.mlp_loss_grad(tn.params, x, y, grad, tensor_cores=tc)
        a.record()
        for _ in range(10):
            holder.mlp_loss_grad(tn.params, x, y, grad, tensor_cores=tc)
        b.record()
        torch.cuda.synchronize()
        res[tc] = (last, acc, mae, a.elapsed_time(b) / 10)
        assert holder.stats()["tensor_timeouts"] == 0
        holder.close()
    print("training: CUDA cores loss %.4f top-1 %.4f grad %.3f ms; tensor cores loss %.4f top-1 %.4f grad %.3f ms"
          " (%d rows)" % (res[False][0], res[False][1], res[False][3], res[True][0], res[True][1], res[True][3],
                          x.shape[0]))
    assert abs(res[True][0] - res[False][0]) <= 0.02 * res[False][0]
    assert abs(res[True][1] - res[False][1]) <= 0.02
