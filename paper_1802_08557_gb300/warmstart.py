"""Learned warm start: train the warm-start network on LPs this library has
solved, and solve new LPs of the same family from its proposal.

The arithmetic runs in the library's kernels (solves, features, labels, the
network's forward/backward/Adam, the warm solve); this module only orders the
calls and holds device buffers (PyTorch tensors).  The family is a set of LPs
of one size m x n that differ in b and c (for example one shared A); the
network maps (b, c) to one logit per constraint, "active at the optimum"."""
from __future__ import annotations

import math

from . import lpbatch as lpb


def batch_features(batch, stream=None):
    """The network's input features (b, c as FP32) of a batch of equal-size
    LPs, as a device tensor (lp_batch_features; no solve)."""
    import torch
    N, m, n = batch.num_lps, int(batch.m[0]), int(batch.n[0])
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64))
    try:
        x = torch.empty((N, m + n), dtype=torch.float32, device="cuda")
        lpb.lp_batch_features(s.h, x, stream)
        torch.cuda.synchronize()
    finally:
        s.close()
    return x


def solved_training_data(batch, stream=None):
    """Solve `batch` cold (FP64) and return device tensors (features, labels)."""
    import torch
    N, m, n = batch.num_lps, int(batch.m[0]), int(batch.n[0])
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64))
    try:
        s.solve(stream)
        x = torch.empty((N, m + n), dtype=torch.float32, device="cuda")
        y = torch.empty((N, m), dtype=torch.float32, device="cuda")
        lpb.lp_batch_features(s.h, x, stream)
        lpb.lp_batch_active_labels(s.h, y, stream)
        torch.cuda.synchronize()
    finally:
        s.close()
    return x, y


def train(batch, epochs: float = 3.0, batch_size: int = 1024, lr: float = 2e-3, lr_final: float = 1e-4,
          pos_weight: float = 4.0, hidden=(512, 512), seed: int = 0, log=None):
    """Train a network on the solved LPs of `batch`; returns (net, info)."""
    N, m, n = batch.num_lps, int(batch.m[0]), int(batch.n[0])
    x, y = solved_training_data(batch)
    net = lpb.Mlp(m + n, hidden[0], hidden[1], m, max_batch=batch_size, seed=seed)
    net.fit_scaling(x)  # per-feature mean and 1/std of the training features, on the GPU
    steps = max(1, int(epochs * N / batch_size))
    first = last = None
    for t in range(steps):
        k = (t * batch_size) % max(1, N - batch_size + 1)
        frac = t / max(1, steps - 1)
        rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))  # cosine decay
        want = t == 0 or t == steps - 1 or (log is not None and t % 200 == 0)
        loss = net.train_step(x[k:k + batch_size], y[k:k + batch_size], rate, pos_weight, want_loss=want)
        if want:
            first = loss if first is None else first
            last = loss
            if log is not None:
                log(f"step {t}/{steps} lr {rate:.2e} loss {loss:.5f}")
    info = {"train_lps": N, "steps": steps, "first_loss": first, "last_loss": last,
            "active_rate": float(y.mean().item())}
    del x, y
    return net, info


def solve_warm(batch, net, threshold: float = 0.2, stream=None):
    """Warm-solve a batch; returns (results dict, plan dict)."""
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64))
    try:
        lpb.lp_batch_solve_warm(s.h, net, threshold, stream)
        r = s.results()
        p = s.plan_info()
    finally:
        s.close()
    return r, p
