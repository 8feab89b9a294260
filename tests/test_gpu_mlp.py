"""GPU kernels of the warm-start network against the network oracle
(oracle/mlp.py), through the C ABI: forward logits, every gradient, one Adam
step, training progress and determinism.

Tolerances.  Both sides round the same operands to BF16; the GPU accumulates
products in FP32 (error ~ K * 2^-24 of the summed magnitudes, K <= 512), the
oracle in FP64.  A hidden activation whose FP32 value lies within that error of
a BF16 rounding boundary can round the other way (one BF16 step, 2^-8
relative) and move the later layers slightly, so gradients are compared per
parameter block in norm (1e-2 relative) rather than element by element, and
logits element by element with a tolerance scaled to their spread."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1802_08557_gb300 import lpbatch as lpb

pytestmark = pytest.mark.gpu

SIZES = (300, 512, 512, 200)


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def unflat(v, sizes):
    out, off = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = v[off:off + o * i].reshape(o, i); off += o * i
        b = v[off:off + o]; off += o
        out.append((W.copy(), b.copy()))
    return out


def _data(batch, sizes, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((batch, sizes[0])).astype(np.float32)
    y = (rng.random((batch, sizes[-1])) < 0.1).astype(np.float32)
    return x, y


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _net_with_oracle_params(sizes, seed, max_batch):
    params = omlp.init_params(sizes, seed=seed)
    rng = np.random.default_rng(seed + 1)
    params = [(W, omlp.bf16_round(rng.standard_normal(b.shape).astype(np.float32) * 0.1)) for W, b in params]
    net = lpb.Mlp(*sizes, max_batch=max_batch, seed=seed)
    net.set_params(flat(params))
    return net, params


@pytest.mark.parametrize("batch", [1, 37, 300])
def test_forward_matches_oracle(batch):
    import torch
    net, params = _net_with_oracle_params(SIZES, seed=4, max_batch=512)
    x, _ = _data(batch, SIZES, seed=batch)
    logits = torch.empty((batch, SIZES[-1]), dtype=torch.float32, device="cuda")
    net.forward(_dev(x), logits)
    torch.cuda.synchronize()
    got = logits.cpu().numpy()
    want, _ = omlp.forward(params, x)
    scale = float(np.std(want)) + 1e-6
    assert np.max(np.abs(got - want)) <= 2e-2 * scale, np.max(np.abs(got - want)) / scale
    assert np.mean(np.abs(got - want)) <= 1e-3 * scale
    net.close()


def test_large_batch_forward_tiled_kernel():
    """Batches whose 128 x 128 tiles fill the GPU take the tiled GEMM (cp.async
    stages, ldmatrix fragments): logits match the oracle, and bit for bit the
    small-tile kernel's on the same rows (forwarded in pieces too small for the
    tiled kernel; each row's result does not depend on the batch)."""
    import torch
    net, params = _net_with_oracle_params(SIZES, seed=5, max_batch=512)
    batch = 6000
    x, _ = _data(batch, SIZES, seed=17)
    dx = _dev(x)
    whole = torch.empty((batch, SIZES[-1]), dtype=torch.float32, device="cuda")
    net.forward(dx, whole)
    pieces = torch.empty_like(whole)
    for r0 in range(0, batch, 1000):
        net.forward(dx[r0:r0 + 1000], pieces[r0:r0 + 1000])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(whole.cpu().numpy(), pieces.cpu().numpy())
    want, _ = omlp.forward(params, x)
    got = whole.cpu().numpy()
    scale = float(np.std(want)) + 1e-6
    assert np.max(np.abs(got - want)) <= 2e-2 * scale
    assert np.mean(np.abs(got - want)) <= 1e-3 * scale
    net.close()


@pytest.mark.parametrize("batch", [64, 250])
def test_gradients_match_oracle(batch):
    net, params = _net_with_oracle_params(SIZES, seed=7, max_batch=256)
    x, y = _data(batch, SIZES, seed=11)
    g, loss = net.gradients(_dev(x), _dev(y), pos_weight=5.0)
    z, cache = omlp.forward(params, x)
    want_loss, g3 = omlp.loss_and_grad_logits(z, y, pos_weight=5.0)
    want = flat(omlp.backward(params, cache, g3))
    assert loss == pytest.approx(want_loss, rel=1e-3)
    got_blocks = unflat(g, SIZES)
    want_blocks = unflat(want, SIZES)
    for li, ((gW, gb), (wW, wb)) in enumerate(zip(got_blocks, want_blocks)):
        for name, a, b in (("W", gW, wW), ("b", gb, wb)):
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel <= 1e-2, f"layer {li + 1} d{name}: relative error {rel:.3e}"
    net.close()


def test_gradients_are_deterministic():
    net, _ = _net_with_oracle_params(SIZES, seed=8, max_batch=128)
    x, y = _data(128, SIZES, seed=3)
    g1, l1 = net.gradients(_dev(x), _dev(y), pos_weight=2.0)
    g2, l2 = net.gradients(_dev(x), _dev(y), pos_weight=2.0)
    np.testing.assert_array_equal(g1, g2)
    assert l1 == l2
    net.close()


def test_adam_step_matches_oracle_update():
    net, params = _net_with_oracle_params(SIZES, seed=9, max_batch=128)
    x, y = _data(96, SIZES, seed=5)
    g, _ = net.gradients(_dev(x), _dev(y), pos_weight=3.0)
    p0 = net.get_params()
    net.train_step(_dev(x), _dev(y), lr=1e-3, pos_weight=3.0)
    p1 = net.get_params()
    grads = unflat(g, SIZES)
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in unflat(p0, SIZES)]
    want, _, _ = omlp.adam_step(unflat(p0, SIZES), grads, zeros, zeros, t=1, lr=1e-3)
    np.testing.assert_allclose(p1, flat(want), rtol=1e-6, atol=1e-7)
    net.close()


def test_training_reduces_loss_on_a_learnable_task():
    """Targets are a fixed random linear threshold of the inputs: a network
    that learns must cut the loss well below its starting value."""
    import torch
    sizes = (40, 64, 64, 16)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4096, sizes[0])).astype(np.float32)
    Wt = rng.standard_normal((sizes[0], sizes[-1])).astype(np.float32)
    y = (x @ Wt > 0.5).astype(np.float32)
    net = lpb.Mlp(*sizes, max_batch=512, seed=1)
    dx, dy = _dev(x), _dev(y)
    first = net.train_step(dx[:512], dy[:512], lr=3e-3, want_loss=True)
    for step in range(300):
        k = (step * 512) % 4096
        net.train_step(dx[k:k + 512], dy[k:k + 512], lr=3e-3)
    last = net.train_step(dx[:512], dy[:512], lr=3e-3, want_loss=True)
    assert last < 0.35 * first, (first, last)
    torch.cuda.synchronize()
    net.close()


def test_errors_are_codes():
    net = lpb.Mlp(8, 16, 16, 4, max_batch=32, seed=0)
    x = np.zeros((8, 8), np.float32)
    y = np.zeros((8, 4), np.float32)
    with pytest.raises(lpb.LPBError) as e:
        net.train_step(x, y, lr=1e-3)              # host memory
    assert e.value.code == lpb.LPB_EINVAL
    with pytest.raises(lpb.LPBError) as e:
        net.train_step(_dev(np.zeros((64, 8), np.float32)), _dev(np.zeros((64, 4), np.float32)), lr=1e-3)
    assert e.value.code == lpb.LPB_EINVAL          # batch > max_batch
    h = lpb.ctypes.c_void_p()
    assert lpb.load().lp_mlp_create(lpb.ctypes.byref(h), 0, 4, 4, 4, 8, 0) == lpb.LPB_EINVAL
    net.close()
