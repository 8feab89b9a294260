"""CPU reference (oracle) of the warm-start network: a 3-layer perceptron
(in -> h1 -> h2 -> out, ReLU) that maps an LP's right-hand side and costs to
one logit per constraint ("is this constraint active at the optimum").  The
paper has no counterpart (its solver always starts from the slack basis); the
network, its precision scheme and its loss are the definition below.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Precision scheme (the CUDA kernels follow it step for step):
  * every matrix product takes BF16 operands (round to nearest even) and
    accumulates in FP32 -- here it is accumulated in FP64, which differs from
    any FP32 order by far less than the test tolerances;
  * biases, pre-activations, the loss and every gradient are FP32 values; an
    operand is rounded to BF16 only where it enters a product;
  * forward:  a1 = bf(x) bf(W1)^T + b1,  h1 = relu(a1)
              a2 = bf(h1) bf(W2)^T + b2, h2 = relu(a2)
              z  = bf(h2) bf(W3)^T + b3                        (logits)
  * loss: mean over the batch and the outputs of the weighted binary cross
    entropy  w_y * softplus(-z) (y = 1) or softplus(z) (y = 0), with w_1 =
    pos_weight and w_0 = 1;
  * backward: g3 = dL/dz = (w * (sigmoid(z) - y)) / (batch * out) with w the
    per-element weight [y*pos_weight + (1-y)];
              dW3 = bf(g3)^T bf(h2),  db3 = sum_batch g3
              g2 = (bf(g3) bf(W3)) * [a2 > 0]
              dW2 = bf(g2)^T bf(h1),  db2 = sum_batch g2
              g1 = (bf(g2) bf(W2)) * [a1 > 0]
              dW1 = bf(g1)^T bf(x),   db1 = sum_batch g1
  * Adam (lr, beta1, beta2, eps, step t) on FP32 master weights.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as
    FP32.  NaN stays NaN; values beyond the BF16 range become infinities."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).copy()
    nan = np.isnan(f)
    out[nan] = f[nan]
    return out


def init_params(sizes, seed: int = 0):
    """He-uniform FP32 weights (BF16-representable) and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fan_in)
        W = bf16_round(rng.uniform(-lim, lim, (fan_out, fan_in)).astype(np.float32))
        params.append((W, np.zeros(fan_out, np.float32)))
    return params


def _mm(a, b):
    """Product of BF16-rounded operands, accumulated in FP64, as FP32."""
    return (bf16_round(a).astype(np.float64) @ bf16_round(b).astype(np.float64)).astype(np.float32)


def forward(params, x):
    """Returns (logits, cache)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    a1 = _mm(x, W1.T) + b1
    h1 = np.maximum(a1, 0.0).astype(np.float32)
    a2 = _mm(h1, W2.T) + b2
    h2 = np.maximum(a2, 0.0).astype(np.float32)
    z = _mm(h2, W3.T) + b3
    return z.astype(np.float32), (x, a1, h1, a2, h2, z)


def loss_and_grad_logits(z, y, pos_weight: float = 1.0):
    """Weighted BCE with logits, mean over every element; and dL/dz."""
    z64 = z.astype(np.float64)
    w = y * pos_weight + (1.0 - y)
    sp_neg = np.logaddexp(0.0, -z64)   # softplus(-z)
    sp_pos = np.logaddexp(0.0, z64)    # softplus(z)
    loss = float(np.mean(w * (y * sp_neg + (1.0 - y) * sp_pos)))
    sig = 1.0 / (1.0 + np.exp(-z64))
    g = (w * (sig - y) / z.size).astype(np.float32)
    return loss, g


def backward(params, cache, g3):
    """Gradients [(dW1, db1), (dW2, db2), (dW3, db3)] from dL/dz."""
    (W1, _), (W2, _), (W3, _) = params
    x, a1, h1, a2, h2, _ = cache
    dW3 = _mm(g3.T, h2)
    db3 = g3.astype(np.float64).sum(axis=0).astype(np.float32)
    g2 = (_mm(g3, W3) * (a2 > 0)).astype(np.float32)
    dW2 = _mm(g2.T, h1)
    db2 = g2.astype(np.float64).sum(axis=0).astype(np.float32)
    g1 = (_mm(g2, W2) * (a1 > 0)).astype(np.float32)
    dW1 = _mm(g1.T, x)
    db1 = g1.astype(np.float64).sum(axis=0).astype(np.float32)
    return [(dW1, db1), (dW2, db2), (dW3, db3)]


def adam_step(params, grads, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on FP32 master weights (in FP64, stored FP32)."""
    out_p, out_m, out_v = [], [], []
    c1 = 1.0 - beta1 ** t
    c2 = 1.0 - beta2 ** t
    for (p_pair, g_pair, m_pair, v_pair) in zip(params, grads, m, v):
        new_p, new_m, new_v = [], [], []
        for p, g, mm, vv in zip(p_pair, g_pair, m_pair, v_pair):
            g64 = g.astype(np.float64)
            mm = beta1 * mm.astype(np.float64) + (1 - beta1) * g64
            vv = beta2 * vv.astype(np.float64) + (1 - beta2) * g64 * g64
            step = lr * (mm / c1) / (np.sqrt(vv / c2) + eps)
            new_p.append((p.astype(np.float64) - step).astype(np.float32))
            new_m.append(mm.astype(np.float32))
            new_v.append(vv.astype(np.float32))
        out_p.append(tuple(new_p))
        out_m.append(tuple(new_m))
        out_v.append(tuple(new_v))
    return out_p, out_m, out_v
