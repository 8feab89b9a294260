"""Element-wise error bounds of the warm-start network's GPU results against
the network oracle (oracle/mlp.py).

The oracle takes BF16 operands, sums products exactly enough (FP64) and
rounds once to FP32; the GPU sums the same BF16 products on the tensor cores
in FP32.  For one product C = A B (K terms per element) the GPU's accumulator
then lies within

    gamma_K * sum_k |a_k||b_k|,   gamma_K = K * 2^-23,

of the exact sum: at most K additions, each off by less than one FP32 unit in
the last place (2^-23 relative) even if the hardware truncates while it
aligns the addends instead of rounding to nearest (2^-24).

A BF16 operand that the GPU computed itself (an activation, a gradient) can
differ from the oracle's where the FP32 value it was rounded from lies within
its error bound of a BF16 rounding boundary: both values then lie in the
interval [bf16(v - e), bf16(v + e)] (rounding is monotonic), so the two
operands differ by at most that interval's width w.  A product whose
operands carry widths wa, wb adds

    sum_k  wa_k (|b_k| + wb_k) + |a_k| wb_k

to the bound.  A ReLU mask whose pre-activation lies within its error bound of
0 can go either way: the masked value then lies anywhere between 0 and the
unmasked one.  Propagating these widths layer by layer gives a bound for every
output element; nothing is compared in norm.

Everything is computed in FP64 from the oracle's own values; no GPU value
enters a bound.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as omlp

U23 = 2.0 ** -23   # one FP32 ulp, relative (truncating accumulation)
U24 = 2.0 ** -24   # FP32 round to nearest, relative


def pad32(v: int) -> int:
    return (v + 31) // 32 * 32


def bf(a) -> np.ndarray:
    return omlp.bf16_round(np.asarray(a, np.float32)).astype(np.float64)


def bf16_range(lo, hi):
    """Smallest and largest BF16 value that rounding to nearest can give for
    an FP32 value in [lo, hi] (FP64 bounds, widened outward to FP32 where the
    interval is not a single point)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    lo32 = lo.astype(np.float32)
    hi32 = hi.astype(np.float32)
    wide = hi > lo
    lo32 = np.where(wide, np.nextafter(lo32, np.float32(-np.inf)), lo32)
    hi32 = np.where(wide, np.nextafter(hi32, np.float32(np.inf)), hi32)
    return bf(lo32), bf(hi32)


def mm_err(a, wa, b, wb, K: int) -> np.ndarray:
    """Bound on |GPU accumulator - oracle _mm(a, b)| per element of a @ b
    (a [M x K'], b [K' x N], the oracle's BF16 operand values; wa, wb their
    widths, arrays or 0); K = the padded K the GPU sums over."""
    A = np.abs(a)
    B = np.abs(b)
    wa = np.broadcast_to(np.asarray(wa, np.float64), A.shape)
    wb = np.broadcast_to(np.asarray(wb, np.float64), B.shape)
    exact = np.abs(a @ b)
    operand = wa @ (B + wb) + A @ wb
    accum = K * U23 * ((A + wa) @ (B + wb))
    # the oracle's own FP64 sum and its final rounding to FP32
    oracle = 2.0 * U24 * exact + K * 2.0 ** -52 * (A @ B)
    return operand + accum + oracle


def bias_err(e_acc, value) -> np.ndarray:
    """Bound after adding an FP32 bias on both sides (one rounding each)."""
    return e_acc * (1.0 + 2.0 * U24) + 2.0 * U24 * np.abs(value)


def relu_operand(a, e_a):
    """The oracle's BF16 operand bf16(relu(a)) and the width of the BF16
    values the GPU can hold for it, its pre-activation being within e_a of a."""
    lo, hi = bf16_range(np.maximum(a - e_a, 0.0), np.maximum(a + e_a, 0.0))
    return bf(np.maximum(a, 0.0)), hi - lo


def masked(t, e_t, pre, e_pre):
    """g = t * [pre > 0] with t within e_t and pre within e_pre of the
    oracle's: returns (oracle g, lower and upper bound of the GPU's g)."""
    on = pre > 0
    g = np.where(on, t, 0.0)
    sure_on = pre - e_pre > 0
    sure_off = pre + e_pre <= 0
    lo = np.where(sure_off, 0.0, t - e_t)
    hi = np.where(sure_off, 0.0, t + e_t)
    amb = ~sure_on & ~sure_off
    lo = np.where(amb, np.minimum(lo, 0.0), lo)
    hi = np.where(amb, np.maximum(hi, 0.0), hi)
    return g, lo, hi


def network_bounds(params, x, y, pos_weight: float, forward_exact: bool = False) -> dict:
    """Oracle values and element-wise bounds of the GPU's results.

    forward_exact=False: the GPU runs the whole network (lp_mlp_forward /
    lp_mlp_gradients); its forward values carry their own errors.
    forward_exact=True: the GPU gets the oracle's a1, a2, z
    (lp_mlp_gradients_at), so only the backward pass adds errors.

    Returns dict with "z", "loss", "dW1", "db1", "dW2", "db2", "dW3", "db3",
    each a pair (oracle value, bound)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    x = np.asarray(x, np.float32)
    batch, n_in = x.shape
    h1n, h2n, n_out = W1.shape[0], W2.shape[0], W3.shape[0]
    z32, cache = omlp.forward(params, x)
    _, a1, _, a2, _, _ = (np.asarray(v, np.float64) for v in cache)
    z = z32.astype(np.float64)
    xo = bf(x)
    W1o, W2o, W3o = bf(W1), bf(W2), bf(W3)
    out = {}

    # ---- forward -----------------------------------------------------------
    if forward_exact:
        e_a1 = np.zeros_like(a1)
        e_a2 = np.zeros_like(a2)
        e_z = np.zeros_like(z)
    else:
        e_a1 = bias_err(mm_err(xo, 0.0, W1o.T, 0.0, pad32(n_in)), a1)
    out["a1"] = (a1, e_a1)
    h1o, w_h1 = relu_operand(a1, e_a1)
    if not forward_exact:
        e_a2 = bias_err(mm_err(h1o, w_h1, W2o.T, 0.0, pad32(h1n)), a2)
    h2o, w_h2 = relu_operand(a2, e_a2)
    if not forward_exact:
        e_z = bias_err(mm_err(h2o, w_h2, W3o.T, 0.0, pad32(h2n)), z)
    out["z"] = (z, e_z)

    # ---- loss and dL/dz ----------------------------------------------------
    loss, g3_32 = omlp.loss_and_grad_logits(z32, y, pos_weight)
    g3 = g3_32.astype(np.float64)
    w = y * pos_weight + (1.0 - y)
    BN = float(z.size)
    # |d sigmoid/dz| <= 1/4; each side rounds to FP32 once; FP64 sigmoid
    # minus a target of 1 cancels (absolute FP64 error of a few 2^-53)
    e_g3 = w * e_z / (4.0 * BN) + 2.0 * U23 * np.abs(g3) + w * 4.0 * 2.0 ** -53 / BN
    e_loss = float(np.sum(w * e_z) / BN) + 1e-10 * abs(loss) + 1e-300
    out["loss"] = (loss, e_loss)
    g3lo, g3hi = bf16_range(g3 - e_g3, g3 + e_g3)
    g3o, w_g3 = bf(g3), g3hi - g3lo

    # the oracle's gradients; the bounds below are built beside them
    (dW1o, db1o), (dW2o, db2o), (dW3o, db3o) = omlp.backward(params, cache, g3_32)
    Kb = pad32(batch)
    # layer 3
    out["dW3"] = (dW3o, mm_err(g3o.T, w_g3.T, h2o, w_h2, Kb))
    out["db3"] = (db3o, e_g3.sum(axis=0) + 2.0 * U24 * np.abs(g3.sum(axis=0))
                  + batch * 2.0 ** -52 * np.abs(g3).sum(axis=0))
    t2 = g3o @ W3o
    e_t2 = mm_err(g3o, w_g3, W3o, 0.0, pad32(n_out))
    g2, g2lo, g2hi = masked(t2, e_t2, a2, e_a2)
    e_g2 = np.maximum(g2hi - g2, g2 - g2lo)
    bl, bh = bf16_range(g2lo, g2hi)
    g2o, w_g2 = bf(g2), bh - bl
    # layer 2
    out["dW2"] = (dW2o, mm_err(g2o.T, w_g2.T, h1o, w_h1, Kb))
    out["db2"] = (db2o, e_g2.sum(axis=0) + 2.0 * U24 * np.abs(g2).sum(axis=0)
                  + batch * 2.0 ** -52 * np.abs(g2).sum(axis=0))
    t1 = g2o @ W2o
    e_t1 = mm_err(g2o, w_g2, W2o, 0.0, pad32(h2n))
    g1, g1lo, g1hi = masked(t1, e_t1, a1, e_a1)
    e_g1 = np.maximum(g1hi - g1, g1 - g1lo)
    bl, bh = bf16_range(g1lo, g1hi)
    g1o, w_g1 = bf(g1), bh - bl
    # layer 1
    out["dW1"] = (dW1o, mm_err(g1o.T, w_g1.T, xo, 0.0, Kb))
    out["db1"] = (db1o, e_g1.sum(axis=0) + 2.0 * U24 * np.abs(g1).sum(axis=0)
                  + batch * 2.0 ** -52 * np.abs(g1).sum(axis=0))
    return out


def check(name, got, want, bound, slack: float = 1.0):
    """Assert |got - want| <= slack * bound + 1e-30 element by element;
    report the worst element."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    bound = np.broadcast_to(np.asarray(bound, np.float64), want.shape)
    assert got.shape == want.shape, (name, got.shape, want.shape)
    assert np.all(np.isfinite(got)), f"{name}: non-finite values"
    err = np.abs(got - want)
    lim = slack * bound + 1e-30
    bad = err > lim
    if bad.any():
        i = np.unravel_index(np.argmax(err - lim), err.shape)
        raise AssertionError(f"{name}: {int(bad.sum())} of {err.size} elements outside their bound; worst at {i}: "
                             f"got {got[i]!r}, oracle {want[i]!r}, |diff| {err[i]:.3e} > bound {lim[i]:.3e}")
    return float(np.max(err / lim))
