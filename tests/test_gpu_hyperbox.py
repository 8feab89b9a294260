"""GPU parity of lp_hyperbox_solve (Section 4.4, Eq. 7) against the hyperbox
oracle, through the C ABI.

x (the maximiser) is a selection and must match bit for bit.  obj is a sum of
dim products: the kernel takes fused multiply-adds in a fixed order, the
oracle rounds each product and then adds, so each is within
dim * 2^-53 * sum_i |l_i h_i| of the exact sum and the two within twice that
(plus one rounding); the test uses that bound.  Integer data is exact on both
sides and must match bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import hyperbox as ohb
from paper_1802_08557_gb300 import lpbatch as lpb

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _inputs(num, dim, seed, per_lp=False):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((num, dim))
    L[rng.random((num, dim)) < 0.05] = 0.0
    shape = (num, dim) if per_lp else (dim,)
    lo = rng.uniform(-3.0, 1.0, shape)
    hi = lo + rng.uniform(0.0, 4.0, shape)
    return L, lo, hi


def _check(L, lo, hi, obj, x):
    want_obj, want_x = ohb.hyperbox_solve(L, lo, hi)
    np.testing.assert_array_equal(x, want_x)
    dim = L.shape[1]
    mag = np.abs(L * want_x).sum(axis=1)
    bound = 2.0 * (dim + 1) * U * mag + 4.0 * U * np.abs(want_obj)
    err = np.abs(obj - want_obj)
    assert np.all(err <= bound), f"max excess {float(np.max(err - bound))}"


def _solve_device(L, lo, hi, per_lp, with_x=True):
    import torch
    dL, dlo, dhi = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (L, lo, hi))
    obj = torch.empty(L.shape[0], dtype=torch.float64, device="cuda")
    x = torch.empty(L.shape, dtype=torch.float64, device="cuda") if with_x else None
    lpb.lp_hyperbox_solve(dL, dlo, dhi, obj, x, box_per_lp=per_lp, ptr_kind=lpb.LPB_DEVICE,
                          stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return obj.cpu().numpy(), (x.cpu().numpy() if with_x else None)


@pytest.mark.parametrize("dim", [1, 2, 5, 28, 63, 64, 65, 300])
@pytest.mark.parametrize("per_lp", [False, True])
def test_parity_tiles_and_ragged_tail(dim, per_lp):
    """Several tiles of 128 (or 64) LPs plus a ragged tail; dim up to the
    tile kernel's limit (64) and beyond it (one warp per LP)."""
    num = 128 * 7 + 37
    L, lo, hi = _inputs(num, dim, seed=dim * 7 + per_lp, per_lp=per_lp)
    obj, x = _solve_device(L, lo, hi, per_lp)
    _check(L, lo, hi, obj, x)


@pytest.mark.parametrize("per_lp", [False, True])
def test_host_pointers_match_device_pointers(per_lp):
    L, lo, hi = _inputs(1000, 28, seed=5, per_lp=per_lp)
    obj_h = np.empty(1000)
    x_h = np.empty((1000, 28))
    lpb.lp_hyperbox_solve(L, lo, hi, obj_h, x_h, box_per_lp=per_lp, ptr_kind=lpb.LPB_HOST)
    obj_d, x_d = _solve_device(L, lo, hi, per_lp)
    np.testing.assert_array_equal(obj_h, obj_d)
    np.testing.assert_array_equal(x_h, x_d)
    _check(L, lo, hi, obj_h, x_h)


@pytest.mark.parametrize("per_lp", [False, True])
def test_unaligned_arrays_take_plain_loads_with_same_bits(per_lp):
    """Arrays 8 bytes off a 16-byte boundary cannot be bulk-copied; the plain
    path must give the same bits (same summation order)."""
    import torch
    num, dim = 128 * 5, 7
    L, lo, hi = _inputs(num, dim, seed=9, per_lp=per_lp)
    ref_obj, ref_x = _solve_device(L, lo, hi, per_lp)

    def shifted(a):
        buf = torch.empty(a.size + 1, dtype=torch.float64, device="cuda")
        buf[1:] = torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
        return buf[1:]

    dL, dlo, dhi = shifted(L), shifted(lo), shifted(hi)
    assert dL.data_ptr() % 16 == 8
    obj = torch.empty(num, dtype=torch.float64, device="cuda")
    x = torch.empty(num * dim, dtype=torch.float64, device="cuda")
    lpb.load().lp_hyperbox_solve(num, dim, dlo.data_ptr(), dhi.data_ptr(), int(per_lp), dL.data_ptr(),
                                 obj.data_ptr(), x.data_ptr(), lpb.LPB_DEVICE, None)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(obj.cpu().numpy(), ref_obj)
    np.testing.assert_array_equal(x.cpu().numpy().reshape(num, dim), ref_x)


def test_integer_data_is_exact():
    rng = np.random.default_rng(17)
    L = rng.integers(-1000, 1001, (5000, 28)).astype(np.float64)
    lo = rng.integers(-100, 1, 28).astype(np.float64)
    hi = lo + rng.integers(0, 200, 28)
    obj, x = _solve_device(L, lo, hi, False)
    want_obj, want_x = ohb.hyperbox_solve(L, lo, hi)
    np.testing.assert_array_equal(obj, want_obj)
    np.testing.assert_array_equal(x, want_x)


def test_zero_and_negative_zero_take_the_upper_bound():
    L = np.array([[0.0, -0.0, 1.0, -1.0]] * 3)
    lo = np.array([-1.0, -2.0, -3.0, -4.0])
    hi = np.array([1.0, 2.0, 3.0, 4.0])
    obj, x = _solve_device(L, lo, hi, False)
    np.testing.assert_array_equal(x, np.tile(np.array([1.0, 2.0, 3.0, -4.0]), (3, 1)))
    np.testing.assert_array_equal(obj, np.full(3, 3.0 + 4.0))


def test_obj_only_and_empty_batch():
    L, lo, hi = _inputs(300, 10, seed=3)
    obj, _ = _solve_device(L, lo, hi, False, with_x=False)
    _check(L, lo, hi, obj, ohb.hyperbox_solve(L, lo, hi)[1])
    lpb.lp_hyperbox_solve(np.zeros((0, 10)), lo, hi, np.zeros(0), None, ptr_kind=lpb.LPB_HOST)


def test_errors_are_codes():
    L, lo, hi = _inputs(10, 4, seed=1)
    obj = np.empty(10)
    lib = lpb.load()
    args = (lo.ctypes.data, hi.ctypes.data, 0, L.ctypes.data, obj.ctypes.data, None, lpb.LPB_HOST, None)
    assert lib.lp_hyperbox_solve(10, 0, *args) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(-1, 4, *args) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(10, (1 << 20) + 1, *args) == lpb.LPB_ETOOBIG
    assert lib.lp_hyperbox_solve(10, 4, lo.ctypes.data, hi.ctypes.data, 0, None, obj.ctypes.data, None,
                                 lpb.LPB_HOST, None) == lpb.LPB_EINVAL
    # host memory passed as device memory is refused before any launch
    with pytest.raises(lpb.LPBError) as e:
        lpb.lp_hyperbox_solve(L, lo, hi, obj, None, ptr_kind=lpb.LPB_DEVICE)
    assert e.value.code == lpb.LPB_EINVAL


@pytest.mark.slow
def test_full_size_sampled():
    """The bench workload (2^22 directions in R^28, one box), in the bench's
    launch configuration; sampled outputs against the oracle."""
    import torch
    from paper_1802_08557_gb300 import workloads as W
    L, lo, hi = W.hyperbox_directions(1 << 22, 28)
    dL = torch.from_numpy(L).cuda()
    dlo, dhi = torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda()
    obj = torch.empty(L.shape[0], dtype=torch.float64, device="cuda")
    lpb.lp_hyperbox_solve(dL, dlo, dhi, obj, None, ptr_kind=lpb.LPB_DEVICE)
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).choice(L.shape[0], 4000, replace=False)
    got = obj.cpu().numpy()[idx]
    want, want_x = ohb.hyperbox_solve(L[idx], lo, hi)
    mag = np.abs(L[idx] * want_x).sum(axis=1)
    assert np.all(np.abs(got - want) <= 2.0 * 29 * U * mag + 4.0 * U * np.abs(want))
