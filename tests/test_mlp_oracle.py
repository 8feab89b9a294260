"""Pins of the warm-start network oracle (oracle/mlp.py) against things other
than itself: BF16 rounding against hand-worked ties and torch's CPU cast,
back-propagation against central finite differences of the loss (with BF16
rounding switched off, so the algebra alone is tested), closed forms of the
loss and of Adam's first step, and a mutation check."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle import mlp

_SRC = os.path.join(os.path.dirname(oracle.__file__), "mlp.py")


def test_bf16_round_ties_and_library_cast():
    one = np.float32(1.0)
    u = 2.0 ** -8
    vals = np.array([1.0, 1 + u, 1 + 3 * u, 1 + 2 * u, -1 - u, 3.0e38, 1e-40, 0.0, -0.0], np.float32)
    got = mlp.bf16_round(vals)
    assert got[0] == one
    assert got[1] == one                       # tie between 1 and 1+2^-7: to even (1)
    assert got[2] == np.float32(1 + 4 * u)     # tie between 1+2^-7 and 1+2^-6: to even
    assert got[3] == np.float32(1 + 2 * u)     # exactly representable
    assert got[4] == -one
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        vals])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def _exact_module():
    """The oracle with BF16 rounding switched off: pure FP32/FP64 algebra."""
    src = open(_SRC).read().replace("def bf16_round(a) -> np.ndarray:",
                                    "def bf16_round(a) -> np.ndarray:\n    return np.asarray(a, np.float32)\n\n\n"
                                    "def _unused(a):")
    ns = {}
    exec(compile(src, "mlp_exact", "exec"), ns)
    return ns


def _fd_check(ns, pos_weight=3.0):
    rng = np.random.default_rng(1)
    sizes = (7, 8, 8, 5)  # equal hidden widths, like 512 -> 512
    params = [(rng.standard_normal((o, i)).astype(np.float32) * 0.5, rng.standard_normal(o).astype(np.float32) * 0.1)
              for i, o in zip(sizes[:-1], sizes[1:])]
    x = rng.standard_normal((6, sizes[0])).astype(np.float32)
    y = (rng.random((6, sizes[-1])) < 0.3).astype(np.float32)

    def loss_of(p):
        z, _ = ns["forward"](p, x)
        return ns["loss_and_grad_logits"](z, y, pos_weight)[0]

    z, cache = ns["forward"](params, x)
    _, g3 = ns["loss_and_grad_logits"](z, y, pos_weight)
    grads = ns["backward"](params, cache, g3)
    h = 1e-3
    for li in range(3):
        for which in range(2):
            base = params[li][which]
            flat_idx = rng.choice(base.size, min(base.size, 12), replace=False)
            for fi in flat_idx:
                idx = np.unravel_index(fi, base.shape)
                pp = [list(t) for t in params]
                plus = base.copy(); plus[idx] += h
                minus = base.copy(); minus[idx] -= h
                pp[li][which] = plus
                lp = loss_of([tuple(t) for t in pp])
                pp[li][which] = minus
                lm = loss_of([tuple(t) for t in pp])
                fd = (lp - lm) / (2 * h)
                an = float(grads[li][which][idx])
                assert abs(fd - an) <= 2e-3 * max(1e-2, abs(fd)), (li, which, idx, fd, an)


def test_backprop_matches_finite_differences():
    _fd_check(_exact_module())


def test_loss_closed_forms():
    z = np.zeros((4, 3), np.float32)
    y = np.array([[1, 0, 1]] * 4, np.float32)
    loss, g = mlp.loss_and_grad_logits(z, y, pos_weight=1.0)
    assert loss == pytest.approx(np.log(2.0), rel=1e-12)
    np.testing.assert_allclose(g, (0.5 - y) / 12.0, rtol=1e-6)
    # positive weight scales the positive terms only
    loss_w, g_w = mlp.loss_and_grad_logits(z, y, pos_weight=4.0)
    assert loss_w == pytest.approx(np.log(2.0) * (8 * 4 + 4) / 12.0, rel=1e-12)
    np.testing.assert_allclose(g_w[:, 0], 4 * (0.5 - 1.0) / 12.0, rtol=1e-6)
    # confident and right: loss ~ 0
    assert mlp.loss_and_grad_logits(np.full((1, 1), 40.0, np.float32), np.ones((1, 1), np.float32))[0] < 1e-15


def test_adam_first_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(2)
    params = mlp.init_params((5, 4, 3, 2), seed=3)
    grads = [(rng.standard_normal(W.shape).astype(np.float32), rng.standard_normal(b.shape).astype(np.float32))
             for W, b in params]
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    new, _, _ = mlp.adam_step(params, grads, zeros, zeros, t=1, lr=0.01, eps=1e-12)
    for (p0, p1, g) in zip(params, new, grads):
        for a, b, gg in zip(p0, p1, g):
            np.testing.assert_allclose(b - a, -0.01 * np.sign(gg), rtol=1e-5, atol=1e-7)


def test_init_is_bf16_representable_and_scaled():
    params = mlp.init_params((300, 512, 512, 200), seed=0)
    for W, b in params:
        np.testing.assert_array_equal(mlp.bf16_round(W), W)
        assert np.all(b == 0)
        assert abs(W.std() * np.sqrt(W.shape[1]) - np.sqrt(2.0)) < 0.05  # He scale


MUTATIONS = {
    "relu mask dropped": ("g2 = (_mm(g3, W3) * (a2 > 0)).astype(np.float32)", "g2 = _mm(g3, W3).astype(np.float32)"),
    "mask from wrong layer": ("g1 = (_mm(g2, W2) * (a1 > 0)).astype(np.float32)",
                              "g1 = (_mm(g2, W2) * (a2 > 0)).astype(np.float32)"),
    "gradient sign": ("g = (w * (sig - y) / z.size).astype(np.float32)", "g = (w * (y - sig) / z.size).astype(np.float32)"),
    "weight on negatives": ("w = y * pos_weight + (1.0 - y)", "w = (1.0 - y) * pos_weight + y"),
    "bias grad mean": ("db3 = g3.astype(np.float64).sum(axis=0).astype(np.float32)",
                       "db3 = g3.astype(np.float64).mean(axis=0).astype(np.float32)"),
    "weight grad from wrong activation": ("dW2 = _mm(g2.T, h1)", "dW2 = _mm(g2.T, h2)"),
    "hidden activation skipped": ("h2 = np.maximum(a2, 0.0).astype(np.float32)", "h2 = a2.astype(np.float32)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(_SRC).read()
    assert old in src, old
    src = src.replace(old, new).replace("def bf16_round(a) -> np.ndarray:",
                                        "def bf16_round(a) -> np.ndarray:\n    return np.asarray(a, np.float32)\n\n\n"
                                        "def _unused(a):")
    ns = {}
    exec(compile(src, "mlp_mutant", "exec"), ns)
    caught = False
    try:
        _fd_check(ns)
        z = np.zeros((4, 3), np.float32)
        y = np.array([[1, 0, 1]] * 4, np.float32)
        loss, g = ns["loss_and_grad_logits"](z, y, pos_weight=4.0)
        if abs(loss - np.log(2.0) * (8 * 4 + 4) / 12.0) > 1e-9 or not np.allclose(g[:, 0], 4 * (0.5 - 1.0) / 12.0):
            caught = True
    except AssertionError:
        caught = True
    assert caught, f"mutation '{name}' survived the pins"
