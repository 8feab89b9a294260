"""lp_solve_uniform_noalloc, the entry point for callers that must not
allocate device memory while they run (their own pool owns the GPU, or
cudaMalloc/cudaFree would stall a loop), checked against the regular
create/solve/results path on the same data, on two calls in a row, with and
without the optional y output, and across a cudaDeviceReset (the scratch
array's address is looked up in the context of each call).

Both paths run the same per-LP FP64 code, so the results must agree bit for
bit.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    assert len(set(ref["status"].tolist()) & {0, 1, 2}) == 3
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
    for call, with_y in ((0, True), (1, True), (2, False)):
        for t in (status, iters):
            t.fill_(-7)
        for t in (obj, x, y):
            t.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = lpb.lp_solve_uniform_noalloc(N, m, n, A, b, c, status, iters, obj, x, y if with_y else None, None,
                                          stream)
        assert rc == lpb.LPB_OK, f"call {call}: {lpb.strerror(rc)}"
        torch.cuda.synchronize()
        np.testing.assert_array_equal(status.cpu().numpy(), ref["status"], err_msg=f"call {call}")
        np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"], err_msg=f"call {call}")
        np.testing.assert_array_equal(obj.cpu().numpy(), ref["obj"], err_msg=f"call {call}: obj")
        np.testing.assert_array_equal(x.cpu().numpy(), ref["x"], err_msg=f"call {call}: x")
        if with_y:
            np.testing.assert_array_equal(y.cpu().numpy(), ref["y"], err_msg=f"call {call}: y")
        else:
            assert torch.isnan(y).all(), "y was written although NULL was passed"


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
    # only the FP64 kernel runs here: the mixed-precision option is refused
    opts = lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE)
    rc = lpb.lp_solve_uniform_noalloc(1, 5, 5, one, one, one, oi, oi, one, one, None, opts, None)
    assert rc == lpb.LPB_EINVAL


def test_noalloc_after_device_reset(lib, tmp_path):
    """A separate program (this file's companion noalloc_reset.cu linked with
    the library's objects, so both share one CUDA runtime) solves with the
    regular path, with this entry point, resets the device and solves again
    with this entry point in the new context: both calls bit-identical to the
    regular path.  The regular path and lp_solve_host run on both sides of the
    reset too (the library's cached memory pool must start over in the new
    context).  No torch in that process, so nothing else holds the
    context."""
    from paper_1802_08557_gb300 import build
    nvcc = build.nvcc()
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    objs = sorted(os.path.join(build.BUILD_DIR, f) for f in os.listdir(build.BUILD_DIR) if f.endswith(".o"))
    assert objs, "library objects missing"
    exe = tmp_path / "noalloc_reset"
    cmd = [nvcc] + build.ARCH + ["-O2", "-std=c++17", "-I", build.INCLUDE,
                                 os.path.join(ROOT, "tests", "noalloc_reset.cu")] + objs + \
        ["-cudart", "static", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "noalloc reset ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
