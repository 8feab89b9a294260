"""GPU kernels of the warm-start network against the network oracle
(oracle/mlp.py), through the C ABI, element by element: each matrix product
with its epilogue on identical BF16 operands, the backward pass from the
oracle's forward values (layer by layer), the whole network on weights whose
forward pass is exact on both sides, one Adam step, training progress and
determinism.

Bounds (tests/mlp_bounds.py): the GPU accumulates BF16 products in FP32, the
oracle exactly enough in FP64, so each accumulator is within K 2^-23 sum|a||b|
of the oracle's; an operand the GPU rounded to BF16 itself may sit one BF16
step from the oracle's where its FP32 value lies within its own bound of a
rounding boundary, and that width is carried into the next product.  No
block is compared in norm."""
from __future__ import annotations

import numpy as np
import pytest

import mlp_bounds as MB
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


def dyadic_network(sizes, seed, batch):
    """Weights in {-1, 0, 1} 2^-3 with sparse rows, biases and inputs on
    coarse binary grids: every partial sum of the forward pass is exact in
    FP32 in any order and every hidden activation is exact in BF16, so the
    GPU's forward values equal the oracle's bit for bit (asserted from the
    oracle's values below) and only the backward pass rounds."""
    rng = np.random.default_rng(seed)
    params = []
    for (fi, fo), d, bq, br in zip(zip(sizes[:-1], sizes[1:]), (0.05, 0.01, 0.02), (3, 6, 9), (8, 16, 16)):
        W = (rng.choice([-1.0, 0.0, 1.0], size=(fo, fi), p=[d / 2, 1 - d, d / 2]) * 0.125).astype(np.float32)
        b = (rng.integers(-br, br + 1, fo) * 2.0 ** -bq).astype(np.float32)
        params.append((W, b))
    x = rng.integers(-2, 3, (batch, sizes[0])).astype(np.float32)
    y = (rng.random((batch, sizes[-1])) < 0.1).astype(np.float32)
    _, (_, a1, _, a2, _, _) = omlp.forward(params, x)
    for a in (a1, a2):
        r = np.maximum(a, 0.0)
        assert np.array_equal(omlp.bf16_round(r), r), "hidden activations must be exact in BF16"
    return params, x, y


def _check_blocks(got_flat, bounds, sizes, keys=("dW1", "db1", "dW2", "db2", "dW3", "db3")):
    got = unflat(got_flat, sizes)
    named = {"dW1": got[0][0], "db1": got[0][1], "dW2": got[1][0], "db2": got[1][1],
             "dW3": got[2][0], "db3": got[2][1]}
    for k in keys:
        want, bound = bounds[k]
        MB.check(k, named[k], want, bound)


# ---- each product on identical BF16 operands ---------------------------------

def _bf16_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(omlp.bf16_round(a))).to(torch.bfloat16).cuda()


# (M, N, K used, K padded, epilogue): the network's eight products at batch 250
# (K = 300 padded to 320, n_out 200 to 224, batch 250 to 256), and ragged
# small shapes at K = 32, 320, 512
NETWORK_PRODUCTS = [
    ("a1 = x W1^T", 250, 512, 300, 320, lpb.LPB_EPI_BIAS_RELU),
    ("a2 = h1 W2^T", 250, 512, 512, 512, lpb.LPB_EPI_BIAS_RELU),
    ("z = h2 W3^T", 250, 200, 512, 512, lpb.LPB_EPI_BIAS),
    ("dW3 = g3^T h2", 200, 512, 250, 256, lpb.LPB_EPI_STORE),
    ("g2 = g3 W3 * mask", 250, 512, 200, 224, lpb.LPB_EPI_MASK_GRAD),
    ("dW2 = g2^T h1", 512, 512, 250, 256, lpb.LPB_EPI_STORE),
    ("g1 = g2 W2 * mask", 250, 512, 512, 512, lpb.LPB_EPI_MASK_GRAD),
    ("dW1 = g1^T x", 512, 300, 250, 256, lpb.LPB_EPI_STORE),
    ("ragged K=32", 77, 45, 32, 32, lpb.LPB_EPI_BIAS_RELU),
    ("ragged K=320", 130, 200, 300, 320, lpb.LPB_EPI_MASK_GRAD),
    ("ragged K=512", 129, 65, 512, 512, lpb.LPB_EPI_BIAS),
    ("ragged K=32 store", 1, 1, 32, 32, lpb.LPB_EPI_STORE),
]


@pytest.mark.parametrize("form", [lpb.LPB_GEMM_MMA64, lpb.LPB_GEMM_MMA128, lpb.LPB_GEMM_TC],
                         ids=["mma64", "mma128", "tcgen05"])
@pytest.mark.parametrize("case", NETWORK_PRODUCTS, ids=[c[0] for c in NETWORK_PRODUCTS])
def test_product_elementwise(case, form):
    """One product with its epilogue through lp_mlp_gemm_bf16 against the
    oracle's product (_mm) of the same BF16 operands, element by element;
    padding of every output left untouched; h and hT the BF16 rounding of
    the kernel's own FP32 value, bit for bit."""
    import torch
    name, M, N, K, Kp, epi = case
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    lda, ldb = Kp + 8, Kp
    A = np.zeros((M, lda), np.float32)
    A[:, :K] = rng.standard_normal((M, K))
    B = np.zeros((N, ldb), np.float32)
    B[:, :K] = rng.uniform(-0.2, 0.2, (N, K))
    A, B = omlp.bf16_round(A), omlp.bf16_round(B)
    bias = (rng.standard_normal(N) * 0.3).astype(np.float32)
    pre = rng.standard_normal((M, N)).astype(np.float32)
    pre[rng.random((M, N)) < 0.05] = 0.0
    ldc, ldh, ldt = N + 3, N + 5, M + 7
    C = torch.full((M + 1, ldc), float("nan"), dtype=torch.float32, device="cuda")
    pre_d = torch.zeros((M, ldc), dtype=torch.float32, device="cuda")
    pre_d[:, :N] = torch.from_numpy(pre).cuda()
    sentinel = -3072.0  # exact in BF16
    h = torch.full((M + 1, ldh), sentinel, dtype=torch.bfloat16, device="cuda")
    hT = torch.full((N + 1, ldt), sentinel, dtype=torch.bfloat16, device="cuda")
    use_h = epi in (lpb.LPB_EPI_BIAS_RELU, lpb.LPB_EPI_MASK_GRAD)
    lpb.lp_mlp_gemm_bf16(epi, form, M, N, Kp, _bf16_dev(A), lda, _bf16_dev(B), ldb, C, ldc,
                         _dev(bias), pre_d, h if use_h else None, ldh, hT if use_h else None, ldt)
    torch.cuda.synchronize()
    Cn = C.cpu().numpy()
    got = Cn[:M, :N].astype(np.float64)
    assert np.isnan(Cn[M]).all() and np.isnan(Cn[:, N:]).all(), "C written outside [M x N]"
    acc = omlp._mm(A[:, :Kp], B[:, :Kp].T).astype(np.float64)
    e = MB.mm_err(A[:, :Kp].astype(np.float64), 0.0, B[:, :Kp].T.astype(np.float64), 0.0, Kp)
    if epi == lpb.LPB_EPI_STORE:
        want, bound = acc, e
    elif epi in (lpb.LPB_EPI_BIAS, lpb.LPB_EPI_BIAS_RELU):
        want = (acc.astype(np.float32) + bias).astype(np.float64)
        bound = MB.bias_err(e, want)
    else:
        want = np.where(pre > 0, acc, 0.0)
        bound = np.where(pre > 0, e, 0.0)
    MB.check(name, got, want, bound)
    if use_h:
        hn = h.float().cpu().numpy()
        hTn = hT.float().cpu().numpy()
        assert (hn[M] == sentinel).all() and (hn[:, N:] == sentinel).all(), "h written outside [M x N]"
        assert (hTn[N] == sentinel).all() and (hTn[:, M:] == sentinel).all(), "hT written outside [N x M]"
        own = np.maximum(got, 0.0) if epi == lpb.LPB_EPI_BIAS_RELU else got
        np.testing.assert_array_equal(hn[:M, :N], omlp.bf16_round(own.astype(np.float32)))
        np.testing.assert_array_equal(hTn[:N, :M], hn[:M, :N].T)
    assert lpb.lp_mlp_tc_faults() == 0


def test_tcgen05_product_aligned_rows_and_tail_tiles():
    """The tcgen05 kernel's 16-byte epilogue path (rows 16-byte aligned: ldc a
    multiple of 4, ldh of 8) on a product with full and partial 128 x 128
    tiles, in the three epilogues that write h, against the oracle's product;
    h bit for bit the BF16 rounding of the kernel's own FP32 value."""
    import torch
    rng = np.random.default_rng(42)
    M, N, K = 1000, 200, 320
    A = omlp.bf16_round(rng.standard_normal((M, K)).astype(np.float32))
    B = omlp.bf16_round(rng.uniform(-0.2, 0.2, (N, K)).astype(np.float32))
    bias = (rng.standard_normal(N) * 0.3).astype(np.float32)
    pre = rng.standard_normal((M, N)).astype(np.float32)
    acc = omlp._mm(A, B.T).astype(np.float64)
    e = MB.mm_err(A.astype(np.float64), 0.0, B.T.astype(np.float64), 0.0, K)
    for epi in (lpb.LPB_EPI_BIAS_RELU, lpb.LPB_EPI_MASK_GRAD, lpb.LPB_EPI_BIAS):
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        h = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
        hT = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
        use_h = epi != lpb.LPB_EPI_BIAS
        lpb.lp_mlp_gemm_bf16(epi, lpb.LPB_GEMM_TC, M, N, K, _bf16_dev(A), K, _bf16_dev(B), K, C, N, _dev(bias),
                             _dev(pre), h if use_h else None, N, hT if use_h else None, M)
        torch.cuda.synchronize()
        got = C.cpu().numpy().astype(np.float64)
        if epi == lpb.LPB_EPI_MASK_GRAD:
            want, bound = np.where(pre > 0, acc, 0.0), np.where(pre > 0, e, 0.0)
        else:
            want = (acc.astype(np.float32) + bias).astype(np.float64)
            bound = MB.bias_err(e, want)
        MB.check(f"epilogue {epi}", got, want, bound)
        if use_h:
            own = np.maximum(got, 0.0) if epi == lpb.LPB_EPI_BIAS_RELU else got
            hn = h.float().cpu().numpy()
            np.testing.assert_array_equal(hn, omlp.bf16_round(own.astype(np.float32)))
            np.testing.assert_array_equal(hT.float().cpu().numpy(), hn.T)
        if epi == lpb.LPB_EPI_BIAS_RELU:
            # the inference form (no FP32 output, no transposed copy: narrower
            # epilogue staging and a deeper operand ring) writes the same h
            h2 = torch.full((M, N), -3072.0, dtype=torch.bfloat16, device="cuda")
            lpb.lp_mlp_gemm_bf16(epi, lpb.LPB_GEMM_TC, M, N, K, _bf16_dev(A), K, _bf16_dev(B), K, None, 0,
                                 _dev(bias), None, h2, N, None, 0)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(h2.float().cpu().numpy(), hn)
    assert lpb.lp_mlp_tc_faults() == 0


def test_product_argument_errors():
    import torch
    z = torch.zeros((64, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(lpb.LPBError) as e:      # K not a multiple of 32
        lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_STORE, 0, 64, 64, 48, z, 64, z, 64, C, 64)
    assert e.value.code == lpb.LPB_EINVAL
    with pytest.raises(lpb.LPBError) as e:      # bias missing
        lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_BIAS, 0, 64, 64, 64, z, 64, z, 64, C, 64)
    assert e.value.code == lpb.LPB_EINVAL
    with pytest.raises(lpb.LPBError) as e:      # host memory
        lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_STORE, 0, 4, 4, 32, np.zeros((4, 32), np.uint16), 32,
                             np.zeros((4, 32), np.uint16), 32, np.zeros((4, 4), np.float32), 4)
    assert e.value.code == lpb.LPB_EINVAL
    with pytest.raises(lpb.LPBError) as e:      # unknown form
        lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_STORE, 99, 64, 64, 64, z, 64, z, 64, C, 64)
    assert e.value.code == lpb.LPB_EINVAL


# ---- the network -----------------------------------------------------------------

@pytest.mark.parametrize("batch", [1, 37, 300])
def test_forward_exact_network_bitwise(batch):
    """On a network whose forward pass is exact on both sides the logits equal
    the oracle's bit for bit (every product, bias and ReLU of lp_mlp_forward
    checked at once, in both GEMM forms for the larger batch sizes)."""
    import torch
    params, x, _ = dyadic_network(SIZES, seed=batch, batch=batch)
    net = lpb.Mlp(*SIZES, max_batch=512, seed=0)
    net.set_params(flat(params))
    logits = torch.empty((batch, SIZES[-1]), dtype=torch.float32, device="cuda")
    net.forward(_dev(x), logits)
    torch.cuda.synchronize()
    want, _ = omlp.forward(params, x)
    np.testing.assert_array_equal(logits.cpu().numpy(), want)
    net.close()


def test_large_batch_forward_in_one_and_in_pieces():
    """A 6000-row forward (many 128 x 128 tiles per product) gives the same
    logits bit for bit as the same rows forwarded in pieces of 1000 (a row's
    result does not depend on the batch or the tile it lands in), and, on an
    exact network, bit for bit the oracle's."""
    import torch
    for kind in ("random", "exact"):
        batch = 6000
        if kind == "random":
            net, params = _net_with_oracle_params(SIZES, seed=5, max_batch=512)
            x, _ = _data(batch, SIZES, seed=17)
        else:
            params, x, _ = dyadic_network(SIZES, seed=23, batch=batch)
            net = lpb.Mlp(*SIZES, max_batch=512, seed=0)
            net.set_params(flat(params))
        dx = _dev(x)
        whole = torch.empty((batch, SIZES[-1]), dtype=torch.float32, device="cuda")
        net.forward(dx, whole)
        pieces = torch.empty_like(whole)
        for r0 in range(0, batch, 1000):
            net.forward(dx[r0:r0 + 1000], pieces[r0:r0 + 1000])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(whole.cpu().numpy(), pieces.cpu().numpy())
        if kind == "exact":
            want, _ = omlp.forward(params, x)
            np.testing.assert_array_equal(whole.cpu().numpy(), want)
        net.close()


@pytest.mark.parametrize("batch", [64, 250])
def test_gradients_layerwise_elementwise(batch):
    """lp_mlp_gradients_at from the oracle's own forward values (x, a1, a2,
    z): the loss and every gradient element within its propagated bound."""
    net, params = _net_with_oracle_params(SIZES, seed=7, max_batch=256)
    x, y = _data(batch, SIZES, seed=11)
    _, (_, a1, _, a2, _, z) = omlp.forward(params, x)
    g, loss = net.gradients_at(_dev(x), _dev(a1), _dev(a2), _dev(z), _dev(y), pos_weight=5.0)
    bounds = MB.network_bounds(params, x, y.astype(np.float64), 5.0, forward_exact=True)
    want_loss, e_loss = bounds["loss"]
    assert abs(loss - want_loss) <= e_loss, (loss, want_loss)
    _check_blocks(g, bounds, SIZES)
    net.close()


@pytest.mark.parametrize("batch", [64, 250])
def test_gradients_whole_network_elementwise(batch):
    """lp_mlp_gradients (forward and backward in one call) on a network whose
    forward pass is exact: the loss and every gradient element within the
    backward pass's propagated bound."""
    params, x, y = dyadic_network(SIZES, seed=100 + batch, batch=batch)
    net = lpb.Mlp(*SIZES, max_batch=256, seed=0)
    net.set_params(flat(params))
    g, loss = net.gradients(_dev(x), _dev(y), pos_weight=3.0)
    bounds = MB.network_bounds(params, x, y.astype(np.float64), 3.0, forward_exact=True)
    want_loss, e_loss = bounds["loss"]
    assert abs(loss - want_loss) <= e_loss, (loss, want_loss)
    _check_blocks(g, bounds, SIZES)
    net.close()


def test_fit_scaling_is_mean_and_inverse_std_per_feature():
    """lp_mlp_fit_scaling: per-feature mean and 1/std (population) of device
    features, against numpy in FP64 on the same FP32 values; a constant
    feature gets scale 1; the same bits on a repeat call; the scaled
    features have mean 0 and std 1."""
    rng = np.random.default_rng(3)
    rows, n_in = 50_000, 30
    x = (rng.standard_normal((rows, n_in)) * rng.uniform(0.1, 50, n_in) + rng.uniform(-5, 5, n_in)).astype(np.float32)
    x[:, 7] = 0.25
    net = lpb.Mlp(n_in, 16, 16, 4, max_batch=64, seed=0)
    dx = _dev(x)
    net.fit_scaling(dx)
    mean, inv = net.get_scaling()
    f = x.astype(np.float64)
    want_mean = f.mean(axis=0)
    std = f.std(axis=0)
    np.testing.assert_allclose(mean, want_mean.astype(np.float32), rtol=1e-6, atol=1e-7)
    ok = std > 0
    np.testing.assert_allclose(inv[ok], (1.0 / std[ok]).astype(np.float32), rtol=1e-6)
    assert mean[7] == np.float32(0.25) and inv[7] == 1.0
    net.fit_scaling(dx)
    m2, i2 = net.get_scaling()
    np.testing.assert_array_equal(m2, mean)
    np.testing.assert_array_equal(i2, inv)
    z = (f - mean) * inv
    np.testing.assert_allclose(z[:, ok].mean(axis=0), 0.0, atol=1e-5)
    np.testing.assert_allclose(z[:, ok].std(axis=0), 1.0, rtol=1e-5)
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
