"""Pins for the CPU reference of the proposal network (no GPU).

The reference is checked against things other than itself: PyTorch's CPU autograd
in float64 (a library routine for the same layers), central finite differences,
closed forms of the zero network, torch.optim.Adam, and hand values of BF16
rounding plus PyTorch's own float -> bfloat16 conversion.
"""
import math

import numpy as np
import pytest

from oracle import mlp_ref as M

torch = pytest.importorskip("torch")


def _batch(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, M.N_IN)).astype(np.float32)
    slot = rng.integers(0, M.N_SLOTS, size=rows)
    conflict = rng.integers(1, 12, size=rows)
    return X, slot, conflict


def test_sizes():
    assert M.N_PARAMS == 7442
    th = np.arange(M.N_PARAMS, dtype=np.float32)
    W1, b1, W2, b2, W3, b3 = M.unpack(th)
    assert W1.shape == (64, 32) and W1[0, 0] == 0 and b1[0] == 2048
    assert W2[0, 0] == 2112 and b2[0] == 6208 and W3[0, 0] == 6272 and b3[-1] == 7441


def test_bf16_round_hand_values():
    one = 1.0
    vals = np.array([one, one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -8 + 2 ** -20,
                     -2.5, 0.0, -0.0, 3.0e38, float("inf")], dtype=np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7 and goes to the even one (1);
    # 1 + 3*2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even);
    # 3e38 = 1.7632 * 2^127 and 1.7632 * 128 = 225.7 rounds to 226: 226/128 * 2^127
    want = np.array([one, one, one + 2 ** -6, one + 2 ** -7, -2.5, 0.0, -0.0, 226 / 128 * 2.0 ** 127,
                     float("inf")], dtype=np.float32)
    got = M.bf16_round(vals)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (got, want)
    assert np.isnan(M.bf16_round(np.array([np.nan], np.float32)))[0]


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(x).view(np.uint32), t.view(np.uint32))
    assert np.array_equal(M.from_bf16_bits(M.bf16_bits(x)), M.bf16_round(x))


def _torch_loss(theta64, X, slot, conflict, lam):
    th = torch.tensor(theta64, dtype=torch.float64, requires_grad=True)
    W1, b1, W2, b2, W3, b3 = [t for t in M.unpack(th)]
    x = torch.tensor(X, dtype=torch.float64)
    h = torch.relu(torch.nn.functional.linear(x, W1, b1))
    h = torch.relu(torch.nn.functional.linear(h, W2, b2))
    out = torch.nn.functional.linear(h, W3, b3)
    ce = torch.nn.functional.cross_entropy(out[:, :17], torch.tensor(slot, dtype=torch.long))
    tgt = torch.log2(torch.tensor(conflict, dtype=torch.float64))
    loss = ce + lam * torch.mean((out[:, 17] - tgt) ** 2)
    loss.backward()
    return loss.item(), th.grad.numpy(), out.detach().numpy()


def test_forward_backward_match_torch_autograd():
    X, slot, conflict = _batch(257, 1)
    theta = M.bf16_round(M.init_params(5) + np.float32(0.01))
    lam = 0.5
    lt, gt, ot = _torch_loss(theta.astype(np.float64), X, slot, conflict, lam)
    out, _ = M.forward(theta, X, np.float64)
    assert np.allclose(out, ot, rtol=1e-12, atol=1e-12)
    l64, g64 = M.loss_and_grad(theta, X, slot, conflict, lam, np.float64)
    assert abs(l64 - lt) < 1e-12 * max(1.0, abs(lt))
    assert np.allclose(g64, gt, rtol=1e-10, atol=1e-13)
    # the float32 reference stays within float32 rounding of it
    l32, g32 = M.loss_and_grad(theta, X, slot, conflict, lam, np.float32)
    assert abs(l32 - lt) < 1e-5 * abs(lt)
    assert np.max(np.abs(g32 - gt)) < 1e-5 * np.max(np.abs(gt))


def test_finite_differences():
    X, slot, conflict = _batch(16, 2)
    theta = M.init_params(6).astype(np.float64) * 0.7 + 0.003
    lam = 0.3
    _, g = M.loss_and_grad(theta, X, slot, conflict, lam, np.float64)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(M.N_PARAMS, 150, replace=False), [2048, 6208, 7424, 7441]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = M.loss_and_grad(tp, X, slot, conflict, lam, np.float64)
        lm, _ = M.loss_and_grad(tm, X, slot, conflict, lam, np.float64)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_zero_network_closed_form():
    X, slot, conflict = _batch(100, 3)
    theta = np.zeros(M.N_PARAMS, dtype=np.float64)
    lam = 0.25
    loss, g = M.loss_and_grad(theta, X, slot, conflict, lam, np.float64)
    t = np.log2(conflict.astype(np.float64))
    assert abs(loss - (math.log(17) + lam * np.mean(t * t))) < 1e-12
    gb3 = M.unpack(g)[5]
    frac = np.bincount(slot, minlength=17) / 100.0
    assert np.allclose(gb3[:17], 1.0 / 17 - frac, atol=1e-14)
    assert abs(gb3[17] - np.mean(2 * lam * (0 - t))) < 1e-12
    # zero weights block every other gradient
    assert np.all(M.unpack(g)[0] == 0) and np.all(M.unpack(g)[2] == 0) and np.all(M.unpack(g)[4] == 0)


def test_adam_matches_torch():
    rng = np.random.default_rng(9)
    master = rng.standard_normal(M.N_PARAMS)
    ref = torch.tensor(master.copy(), requires_grad=True)
    opt = torch.optim.Adam([ref], lr=3e-3, betas=(0.9, 0.99), eps=1e-7)
    m = np.zeros_like(master)
    v = np.zeros_like(master)
    for t in range(1, 5):
        g = rng.standard_normal(M.N_PARAMS)
        M.adam_step(master, g, m, v, t, 3e-3, 0.9, 0.99, 1e-7)
        ref.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(master, ref.detach().numpy(), rtol=1e-12, atol=1e-12)
