"""CPU reference of the learned locate proposal's network — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
this module.  It shares no code with the CUDA path.

The paper has no learned component; this network is the library's own extension
of the locate step (Section IV, insertion: the walk that finds the triangle holding
the new position).  Its definition is the one ``include/kdt.h`` states:

* 32 input features -> 64 (ReLU) -> 64 (ReLU) -> 18 outputs; outputs 0..16 are the
  logits of the landing slot, output 17 predicts log2(conflict size).
* Parameters, one flat vector of 7442 values in this order: W1 (64 x 32, row =
  output unit), b1 (64), W2 (64 x 64), b2 (64), W3 (18 x 64), b3 (18).
* The network computes with the BF16 values of its parameters (round to nearest,
  ties to even), products and sums in FP32.
* Loss of a batch: mean over rows of cross-entropy(logits, slot) +
  lam * (out17 - log2(conflict))^2.
* Optimiser: Adam (Kingma and Ba, 2015, Algorithm 1) on FP32 master parameters;
  the network then uses their BF16 rounding.

Everything here is plain numpy, layer by layer, in the precision asked for
(float32 for the reference the GPU is compared with, float64 for finite
differences).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT, N_SLOTS = 32, 64, 18, 17
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 7442


def unpack(theta):
    """Views of the flat parameter vector as (W1, b1, W2, b2, W3, b3)."""
    out, o = [], 0
    for _, s in SIZES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def bf16_round(x):
    """Round float32 values to the nearest BF16 value, ties to even (returned as float32).

    BF16 keeps the upper 16 bits of the IEEE binary32 pattern; rounding adds half of
    the dropped range, plus one when the kept part is odd, before truncating.
    Infinities stay; NaNs stay NaN.
    """
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out).astype(np.float32)


def bf16_bits(x):
    """The 16-bit BF16 patterns of bf16_round(x) (uint16)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def init_params(seed: int = 0):
    """He-uniform initial FP32 master parameters (biases zero)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(N_PARAMS, dtype=np.float32)
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    for W in (W1, W2, W3):
        lim = np.sqrt(6.0 / W.shape[1])
        W[...] = rng.uniform(-lim, lim, size=W.shape).astype(np.float32)
    return theta


def forward(theta, X, dtype=np.float32):
    """Outputs (rows x 18) and the activations backward needs.

    theta is used as given: pass bf16_round(master) for the network's BF16 weights."""
    th = np.asarray(theta, dtype=dtype)
    W1, b1, W2, b2, W3, b3 = unpack(th)
    X = np.asarray(X, dtype=dtype)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    out = h2 @ W3.T + b3
    return out, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, slot, conflict, lam, dtype=np.float32):
    """Mean loss over the rows and its gradient with respect to theta (flat)."""
    out, (X, z1, h1, z2, h2) = forward(theta, X, dtype)
    th = np.asarray(theta, dtype=dtype)
    W1, b1, W2, b2, W3, b3 = unpack(th)
    rows = X.shape[0]
    slot = np.asarray(slot, dtype=np.int64)
    target = np.log2(np.asarray(conflict, dtype=dtype)).astype(dtype)
    logits = out[:, :N_SLOTS]
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    s = e.sum(axis=1, keepdims=True)
    logp = logits - mx - np.log(s)
    ce = -logp[np.arange(rows), slot]
    r = out[:, N_SLOTS] - target
    loss = (ce + lam * r * r).mean(dtype=dtype)
    # backward, layer by layer
    dout = np.zeros_like(out)
    dout[:, :N_SLOTS] = e / s
    dout[np.arange(rows), slot] -= 1
    dout[:, N_SLOTS] = 2 * lam * r
    dout /= dtype(rows)
    gW3 = dout.T @ h2
    gb3 = dout.sum(axis=0)
    dh2 = (dout @ W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)]).astype(dtype)
    return dtype(loss), g


def adam_step(master, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place (t counts from 1): biased moments, bias-corrected step."""
    m *= beta1
    m += (1 - beta1) * grad
    v *= beta2
    v += (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    master -= (lr * mhat / (np.sqrt(vhat) + eps)).astype(master.dtype)
    return master


def predict_slot(theta, X):
    """Arg-max slot (lowest index on ties) of each row."""
    out, _ = forward(theta, X)
    return np.argmax(out[:, :N_SLOTS], axis=1)
