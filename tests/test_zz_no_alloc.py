"""lp_solve_uniform_noalloc, the entry point for callers that must not
allocate device memory while they run (their own pool owns the GPU, or
cudaMalloc/cudaFree would stall a loop), checked against the regular
create/solve/results path on the same data, on two calls in a row.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lib():
    from paper_1802_08557_gb300 import build, lpbatch as lpb
    build.build()
    lpb.load()
    return lpb


def _regular(lpb, batch):
    s = lpb.BatchSolver(batch, device_data=True)
    try:
        s.solve()
        return s.results()
    finally:
        s.close()


def test_noalloc_matches_regular_entry_point_on_two_calls(lib):
    import torch
    from paper_1802_08557_gb300 import workloads as W
    lpb = lib
    N, m, n = 1500, 50, 50
    batch = W.mixed_sign_dense(N, m, n, start=4321)  # packed, phase I and every status
    ref = _regular(lpb, batch)
    dev = torch.device("cuda")
    A = torch.from_numpy(batch.A).to(dev)
    b = torch.from_numpy(batch.b).to(dev)
    c = torch.from_numpy(batch.c).to(dev)
    status = torch.empty(N, dtype=torch.int32, device=dev)
    iters = torch.empty(N, dtype=torch.int32, device=dev)
    obj = torch.empty(N, dtype=torch.float64, device=dev)
    x = torch.empty(N * n, dtype=torch.float64, device=dev)
    y = torch.empty(N * m, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        for t in (status, iters):
            t.fill_(-7)
        for t in (obj, x, y):
            t.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = lpb.lp_solve_uniform_noalloc(N, m, n, A, b, c, status, iters, obj, x, y, None, stream)
        assert rc == lpb.LPB_OK, f"call {call}: {lpb.strerror(rc)}"
        torch.cuda.synchronize()
        np.testing.assert_array_equal(status.cpu().numpy(), ref["status"], err_msg=f"call {call}")
        np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"], err_msg=f"call {call}")
        for name, got, want in (("obj", obj, ref["obj"]), ("x", x, ref["x"]), ("y", y, ref["y"])):
            got = got.cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=RTOL, atol=RTOL * max(1.0, float(np.abs(want).max())),
                                       err_msg=f"call {call}: {name}")


def test_noalloc_rejects_batches_beyond_its_scratch(lib):
    import torch
    lpb = lib
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    oi = torch.zeros(1, dtype=torch.int32, device="cuda")
    # one 16384 x 16384 tableau alone is far above the fixed scratch
    rc = lpb.lp_solve_uniform_noalloc(1, 16384, 16384, one, one, one, oi, oi, one, one, None, None, None)
    assert rc == lpb.LPB_ETOOBIG
    # too many LPs for the per-LP descriptors
    rc = lpb.lp_solve_uniform_noalloc(3_000_000, 5, 5, one, one, one, oi, oi, one, one, None, None, None)
    assert rc == lpb.LPB_ETOOBIG
    rc = lpb.lp_solve_uniform_noalloc(0, 5, 5, one, one, one, oi, oi, one, one, None, None, None)
    assert rc == lpb.LPB_EINVAL
