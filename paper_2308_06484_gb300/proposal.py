"""Training and evaluation of the learned locate proposal (this library's extension).

The network, its inputs and its labels are defined with ``kdt_set_trace`` in
``include/kdt.h``.  Everything that computes runs in the library's kernels:
training rows are written by the kinetic kernel while it moves points, the forward
and backward passes and the Adam step are ``kdt_mlp_*`` calls.  This module only
allocates device buffers, draws the seeded initial parameters and the per-epoch row
order, and strings the calls together.
"""
from __future__ import annotations

import math

import numpy as np

from . import kdt as _kdt

MLP_IN, MLP_OUT, MLP_SLOTS, MLP_PARAMS = _kdt.MLP_IN, _kdt.MLP_OUT, _kdt.MLP_SLOTS, _kdt.MLP_PARAMS
_SHAPES = [(64, 32), (64,), (64, 64), (64,), (18, 64), (18,)]


def init_master(seed: int = 0) -> np.ndarray:
    """He-uniform FP32 weights (fan-in), zero biases, as one flat array."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in _SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s).astype(np.float32).ravel())
        else:
            parts.append(np.zeros(s, dtype=np.float32))
    out = np.concatenate(parts)
    assert out.size == MLP_PARAMS
    return out


class Trace:
    """Device buffers the kinetic kernel fills with training rows."""

    def __init__(self, cap: int, device="cuda"):
        import torch
        self.x = torch.zeros((cap, MLP_IN), dtype=torch.float32, device=device)
        self.y = torch.zeros((cap, 2), dtype=torch.int32, device=device)
        self.rows = 0

    def attach(self, tri):
        tri.set_trace(self.x, self.y)

    def detach(self, tri):
        self.rows = tri.trace_count()
        tri.set_trace()
        return self.rows

    def view(self):
        return self.x[: self.rows], self.y[: self.rows]


class Trainer:
    """Adam on FP32 master parameters; the network always runs on their BF16 rounding."""

    def __init__(self, tri, seed: int = 0, lr: float = 2e-3, lam: float = 0.25, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, tensor_cores: bool = False):
        import torch
        self.tri, self.lr, self.lam, self.tensor_cores = tri, lr, lam, tensor_cores
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        dev = "cuda"
        self.master = torch.from_numpy(init_master(seed)).to(dev)
        self.m = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.v = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.grad = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.params = torch.zeros(MLP_PARAMS, dtype=torch.int16, device=dev)
        self.t = 0
        # BF16 rounding of the initial masters: an Adam call with a zero gradient and lr 0
        tri.mlp_adam(self.master, self.grad, self.m, self.v, 1, 0.0, beta1, beta2, eps, self.params)

    def step(self, x, y, index=None):
        """One Adam step on the batch (rows of x / y, or those listed in index)."""
        self.t += 1
        self.tri.mlp_loss_grad(self.params, x, y, self.grad, self.loss, index=index, lam=self.lam,
                               tensor_cores=self.tensor_cores)
        self.tri.mlp_adam(self.master, self.grad, self.m, self.v, self.t, self.lr, self.beta1, self.beta2,
                          self.eps, self.params)

    def fit(self, x, y, epochs: int = 3, batch: int = 8192, seed: int = 0):
        """Mini-batch epochs over the rows in a seeded order; returns the last batch loss."""
        import torch
        n = x.shape[0]
        rng = np.random.default_rng(seed)
        for _ in range(epochs):
            order = torch.from_numpy(rng.permutation(n).astype(np.int64)).to(x.device)
            for s in range(0, n, batch):
                self.step(x, y, order[s:s + batch])
        torch.cuda.synchronize()
        return float(self.loss.item())

    def evaluate(self, x, y):
        """(top-1 slot accuracy, mean absolute error of the log2 cavity) on rows x / y."""
        import torch
        out = torch.empty((x.shape[0], MLP_OUT), dtype=torch.float32, device=x.device)
        self.tri.mlp_forward(self.params, x, out)
        torch.cuda.synchronize()
        pred = torch.argmax(out[:, :MLP_SLOTS], dim=1)
        acc = float((pred == y[:, 0].long()).float().mean().item()) if x.shape[0] else 0.0
        mae = float((out[:, MLP_SLOTS] - torch.log2(y[:, 1].float())).abs().mean().item()) if x.shape[0] else 0.0
        return acc, mae


def collect_traces(sources, cap: int = 1_000_000, bits: int = 24):
    """Training rows of the given workloads: for every (workload, steps) pair, a fresh
    triangulation of the workload's points on its grid records the rows of `steps`
    kinetic steps.  Returns the rows of all sources concatenated (x, y)."""
    import torch
    xs, ys = [], []
    for w, steps in sources:
        tri = _kdt.Triangulation(_kdt.default_config(grid=w.grid, domain_bits=bits))
        tri.build(torch.from_numpy(w.positions).cuda())
        tr = Trace(cap)
        tr.attach(tri)
        for _ in range(steps):
            tri.step(torch.from_numpy(w.next_moves()).cuda())
        tr.detach(tri)
        x, y = tr.view()
        xs.append(x.clone())
        ys.append(y.clone())
        tri.close()
    return torch.cat(xs), torch.cat(ys)


def default_training_sources(c3_n: int = 2_000_000, c3_grid: int = 90, c2_steps: int = 100, c3_steps: int = 4):
    """The training workloads of the proposal: the 1e6-point uniform workload with its
    training seed (102) and the mixture + lattice distribution at c3_n points on a
    c3_grid^2 grid (about 250 points per partition, as the 16e6-point workload) with
    seed 103.  Evaluation uses the uniform workload's own seed (2)."""
    from . import workloads as W
    return [(W.c2(seed=102), c2_steps), (W.c3(n=c3_n, grid=c3_grid, seed=103), c3_steps)]
