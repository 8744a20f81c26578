"""The split-BF16 arithmetic of the tensor-core network kernels, emulated on the CPU
(exact products in float64, each layer's sum rounded once to FP32; the tensor cores
round more often, within the FP32 accumulation term of the bound).  It pins the two
precision choices the kernels make against the oracle's network (oracle/mlp_ref.py):

* inference splits every activation into two BF16 parts: its outputs stay within
  3 * 2^-15 * S3 of the FP64 network (the bound tests/test_gpu_tensor.py applies to
  the kernel) and below 2^-19 * S3 (its check that the second parts are used), where
  BF16 activations alone reach about 2^-14.5 * S3;
* training splits the activations of the row products into three parts and the
  weight-gradient operands into two: the gradients meet the 1e-3 test of the CUDA-core
  kernel, and with two parts in the row products they do not (pre-activations near
  zero land on the other side of the ReLU)."""
import numpy as np
import pytest

from oracle import mlp_ref as M


def _parts(x, n):
    """x as n BF16 parts (hi, then what is left rounded again, ...), float64."""
    out, r = [], np.asarray(x, dtype=np.float32).astype(np.float64)
    for _ in range(n):
        h = M.bf16_round(r.astype(np.float32)).astype(np.float64)
        out.append(h)
        r = r - h
    return out


def _rows(a, w, n):
    """a @ w with a's rows split into n parts and w exact (BF16 weights)."""
    return sum(p @ w for p in _parts(a, n)).astype(np.float32).astype(np.float64)


def _pairs(a, b):
    """a @ b with both operands in two parts, the lo-lo product left out."""
    (ah, al), (bh, bl) = _parts(a, 2), _parts(b, 2)
    return (ah @ bh + ah @ bl + al @ bh).astype(np.float32).astype(np.float64)


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    theta = (M.init_params(seed) * scale + rng.normal(0, 0.02, M.N_PARAMS)).astype(np.float32)
    return M.bf16_round(theta)


def _forward(theta, X, n):
    W1, b1, W2, b2, W3, b3 = [np.asarray(a, np.float64) for a in M.unpack(theta)]
    z1 = _rows(X, W1.T, n) + b1
    h1 = np.maximum(z1, 0)
    z2 = _rows(h1, W2.T, n) + b2
    h2 = np.maximum(z2, 0)
    return _rows(h2, W3.T, n) + b3, (z1, h1, z2, h2)


def _grads(theta, X, slot, conflict, lam, n):
    W1, b1, W2, b2, W3, b3 = [np.asarray(a, np.float64) for a in M.unpack(theta)]
    rows = X.shape[0]
    out, (z1, h1, z2, h2) = _forward(theta, X, n)
    lg = out[:, :17]
    e = np.exp(lg - lg.max(axis=1, keepdims=True))
    dout = np.zeros_like(out)
    dout[:, :17] = e / e.sum(axis=1, keepdims=True)
    dout[np.arange(rows), slot] -= 1
    dout[:, 17] = 2 * lam * (out[:, 17] - np.log2(conflict))
    dout /= rows
    dz2 = _rows(dout, W3, n) * (z2 > 0)
    dz1 = _rows(dz2, W2, n) * (z1 > 0)
    return {"W1": _pairs(dz1.T, X), "W2": _pairs(dz2.T, h1), "W3": _pairs(dout.T, h2)}


def _within_gradient_test(g, gref):
    mx = float(np.max(np.abs(gref)))
    big = np.abs(gref) > 0.05 * mx
    return bool(np.max(np.abs(g - gref)) <= 1e-3 * mx and np.all(np.abs(g - gref)[big] <= 1e-3 * np.abs(gref[big])))


def test_inference_split_meets_the_bound():
    theta = _params(3)
    X = np.random.default_rng(8).standard_normal((4000, 32)).astype(np.float32)
    ref, _ = M.forward(theta, X, np.float64)
    W1, b1, W2, b2, W3, b3 = [np.abs(np.asarray(a, np.float64)) for a in M.unpack(theta)]
    S3 = ((np.abs(X) @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    two, _ = _forward(theta, X, 2)
    one, _ = _forward(theta, X, 1)
    assert np.all(np.abs(two - ref) <= 3 * 2.0 ** -15 * S3)
    # the threshold tests/test_gpu_tensor.py uses to tell the two apart on the kernel's
    # outputs: two parts stay far below it, BF16 activations alone far above it
    assert np.max(np.abs(two - ref) / S3) < 2.0 ** -21
    assert np.max(np.abs(one - ref) / S3) > 2.0 ** -17


def _case(rows, use_index):
    theta = _params(3, scale=0.8)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((rows, 32)).astype(np.float32)
    y = np.stack([rng.integers(0, 17, rows), rng.integers(1, 40, rows)], axis=1).astype(np.int32)
    if use_index:
        sel = np.random.default_rng(5).permutation(rows)[: rows - 7]
        X, y = X[sel], y[sel]
    _, gref = M.loss_and_grad(theta, X, y[:, 0], y[:, 1], 0.25, np.float32)
    ref, o = {}, 0
    for name, shape in M.SIZES:
        k = int(np.prod(shape))
        ref[name] = gref[o:o + k].reshape(shape)
        o += k
    return theta, X, y, ref


@pytest.mark.parametrize("rows,use_index", [(1000, False), (4099, True)])
def test_training_split_meets_the_gradient_test(rows, use_index):
    theta, X, y, ref = _case(rows, use_index)
    g = _grads(theta, X, y[:, 0], y[:, 1], 0.25, 3)
    for name in ("W1", "W2", "W3"):
        assert _within_gradient_test(g[name], ref[name]), name


def test_two_part_rows_fail_the_gradient_test():
    theta, X, y, ref = _case(4099, True)
    g = _grads(theta, X, y[:, 0], y[:, 1], 0.25, 2)
    assert not all(_within_gradient_test(g[n], ref[n]) for n in ("W1", "W2"))
