"""CPU checks of the element-wise bounds (tests/mlp_bounds.py) that the GPU
tests of the warm-start network use.

A numpy stand-in for the GPU pipeline -- BF16 operands, FP32 accumulation in
another order than the oracle's, FP32 epilogues, BF16 activations, the loss
in FP64 -- must stay inside every bound (so the GPU tests do not fail on
rounding), and each of several plausible kernel mistakes planted into the
stand-in must fall outside some bound (so the GPU tests would catch it)."""
from __future__ import annotations

import numpy as np
import pytest

import mlp_bounds as MB
from oracle import mlp as omlp

SIZES = (300, 512, 512, 200)


def _f32mm(a, b, chunk=16, reverse=False):
    """FP32 product accumulated chunk by chunk of K (like the k16 steps of a
    tensor-core kernel), optionally in reverse chunk order."""
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    K = a.shape[1]
    starts = list(range(0, K, chunk))
    if reverse:
        starts = starts[::-1]
    acc = np.zeros((a.shape[0], b.shape[1]), np.float32)
    for k0 in starts:
        acc = (acc + a[:, k0:k0 + chunk] @ b[k0:k0 + chunk]).astype(np.float32)
    return acc


def _bf(a):
    return omlp.bf16_round(np.asarray(a, np.float32))


def stand_in(params, x, y, pw, given=None, mistake=None):
    """The GPU's arithmetic in numpy.  given = (a1, a2, z) skips the forward
    products (lp_mlp_gradients_at).  Returns dict of FP32/FP64 results."""
    (W1, b1), (W2, b2), (W3, b3) = params
    W1b, W2b, W3b = _bf(W1), _bf(W2), _bf(W3)
    xb = _bf(x)
    out = {}
    if given is None:
        acc1 = _f32mm(xb, W1b.T)
        if mistake == "drop_last_k_chunk":
            acc1 = _f32mm(xb[:, :-16], W1b.T[:-16])
        a1 = (acc1 + (b2 if mistake == "wrong_bias" else b1)).astype(np.float32)
        a2 = (_f32mm(_bf(np.maximum(a1, 0)), W2b.T, reverse=True) + b2).astype(np.float32)
        z = (_f32mm(_bf(np.maximum(a2, 0)), W3b.T) + b3).astype(np.float32)
    else:
        a1, a2, z = (np.asarray(v, np.float32) for v in given)
    out["z"] = z
    out["a1"] = a1
    h1 = _bf(np.maximum(a1, 0))
    h2 = _bf(np.maximum(a2, 0))
    z64 = z.astype(np.float64)
    wgt = y * pw + (1.0 - y)
    sp_neg = np.where(z64 > 0, np.log1p(np.exp(-z64)), -z64 + np.log1p(np.exp(z64)))
    out["loss"] = float(np.sum(wgt * (y * sp_neg + (1 - y) * (sp_neg + z64))) / z.size)
    scale = 1.0 if mistake == "no_mean_scale" else 1.0 / z.size
    g3 = (wgt * (1.0 / (1.0 + np.exp(-z64)) - y) * scale).astype(np.float32)
    out["dW3"] = _f32mm(_bf(g3).T, h2)
    out["db3"] = g3.astype(np.float64).sum(axis=0).astype(np.float32)
    mask2 = (a1 if mistake == "mask_from_wrong_layer" else a2) > 0
    g2 = (_f32mm(_bf(g3), W3b) * mask2).astype(np.float32)
    dW2 = _f32mm(_bf(g2).T, h1)
    if mistake == "tile_edge_row":
        dW2 = dW2.copy()
        dW2[63] = dW2[64]
    out["dW2"] = dW2
    out["db2"] = g2.astype(np.float64).sum(axis=0).astype(np.float32)
    g1 = (_f32mm(_bf(g2), W2b) * (a1 > 0)).astype(np.float32)
    dW1 = _f32mm(_bf(g1).T, xb)
    if mistake == "transposed_block":
        dW1 = dW1.copy()
        dW1[:32, :32] = dW1[:32, :32].T
    out["dW1"] = dW1
    out["db1"] = g1.astype(np.float64).sum(axis=0).astype(np.float32)
    return out


def _problem(batch, seed):
    rng = np.random.default_rng(seed)
    params = omlp.init_params(SIZES, seed=seed)
    params = [(W, _bf(rng.standard_normal(b.shape).astype(np.float32) * 0.1)) for W, b in params]
    x = rng.standard_normal((batch, SIZES[0])).astype(np.float32)
    x[:, -7:] = 0.0
    y = (rng.random((batch, SIZES[-1])) < 0.1).astype(np.float64)
    return params, x, y


def _all_within(res, bounds, keys):
    for k in keys:
        want, bound = bounds[k]
        if k == "loss":
            assert abs(res[k] - want) <= bound, (k, res[k], want, bound)
        else:
            MB.check(k, res[k], want, bound)


@pytest.mark.parametrize("batch", [37, 96])
def test_stand_in_within_whole_network_bounds(batch):
    params, x, y = _problem(batch, seed=batch)
    bounds = MB.network_bounds(params, x, y, 4.0, forward_exact=False)
    res = stand_in(params, x, y, 4.0)
    _all_within(res, bounds, ("z", "loss", "dW3", "db3", "dW2", "db2", "dW1", "db1"))


def test_stand_in_within_layerwise_bounds():
    params, x, y = _problem(70, seed=3)
    _, cache = omlp.forward(params, x)
    _, a1, _, a2, _, z = cache
    bounds = MB.network_bounds(params, x, y, 2.0, forward_exact=True)
    res = stand_in(params, x, y, 2.0, given=(a1, a2, z))
    _all_within(res, bounds, ("loss", "dW3", "db3", "dW2", "db2", "dW1", "db1"))


@pytest.mark.parametrize("key,limit", [("dW3", 0.01), ("db3", 0.01), ("dW2", 0.01), ("db2", 0.01),
                                       ("dW1", 0.25), ("db1", 0.05)])
def test_bounds_are_tight_enough_to_mean_something(key, limit):
    """With exact forward values the bounds stay below the stated fraction of
    each block's typical magnitude, so a wrong element (a tile edge, a padded
    column, a transposed copy: errors of the order of the element itself) is
    caught.  dW1 is the loosest: its operand g1 inherits the widths of g2 and
    g3, and a worst-case bound adds every possible BF16 step of them."""
    params, x, y = _problem(64, seed=5)
    bounds = MB.network_bounds(params, x, y, 4.0, forward_exact=True)
    want, bound = bounds[key]
    typical = np.median(np.abs(want[want != 0]))
    assert np.median(bound) < limit * typical, (key, np.median(bound), typical)


@pytest.mark.parametrize("mistake", ["drop_last_k_chunk", "wrong_bias"])
def test_planted_forward_mistakes_leave_the_product_bound(mistake):
    """A product that skips its last 16 K columns, or adds the wrong layer's
    bias, leaves the single-product bound that the GPU product tests use."""
    params, x, y = _problem(64, seed=11)
    x[:, -16:] = np.random.default_rng(1).standard_normal((64, 16)).astype(np.float32)
    bounds = MB.network_bounds(params, x, y, 4.0, forward_exact=False)
    res = stand_in(params, x, y, 4.0, mistake=mistake)
    want, bound = bounds["a1"]
    with pytest.raises(AssertionError):
        MB.check("a1", res["a1"], want, bound)


@pytest.mark.parametrize("mistake,key", [
    ("no_mean_scale", "dW3"),
    ("mask_from_wrong_layer", "dW2"),
    ("tile_edge_row", "dW2"),
    ("transposed_block", "dW1"),
])
def test_planted_backward_mistakes_leave_the_layerwise_bounds(mistake, key):
    """Backward-pass mistakes leave the bounds of the layer-wise and
    exact-forward GPU tests (the forward values are the oracle's)."""
    params, x, y = _problem(64, seed=11)
    _, (_, a1, _, a2, _, z) = omlp.forward(params, x)
    bounds = MB.network_bounds(params, x, y, 4.0, forward_exact=True)
    res = stand_in(params, x, y, 4.0, given=(a1, a2, z), mistake=mistake)
    want, bound = bounds[key]
    with pytest.raises(AssertionError):
        MB.check(key, res[key], want, bound)
