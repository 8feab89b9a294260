"""Helpers shared by the GPU parity tests: run a batch through the C ABI and
through the oracle, and compare element by element."""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_1802_08557_gb300 import lpbatch as lpb

# FP64 parity bar: status and pivot count exact (integer work), objective, x
# and y within 1e-10 relative (the same-pivot-rule FP64 tolerance).
RTOL = 1e-10


def oracle_threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def gpu_solve(batch, device_data=True, opts=None):
    s = lpb.BatchSolver(batch, device_data=device_data, opts=opts)
    try:
        s.solve()
        r = s.results()
        r["plan"] = s.plan_info()
        assert r["plan"]["internal_errors"] == 0, r["plan"]
    finally:
        s.close()
    return r


def oracle_solve(batch, idx=None, opts=None):
    """Oracle results for the LPs ``idx`` (all if None), in the GPU layout."""
    idx = np.arange(batch.num_lps) if idx is None else np.asarray(idx)
    lps = [batch.lp(int(k)) for k in idx]
    oo = None
    if opts is not None:
        oo = oracle.default_opts(eps_opt=opts.eps_opt, eps_piv=opts.eps_piv, eps_feas=opts.eps_feas,
                                 tau=opts.tau, max_iters=opts.max_iters)
    return oracle.solve_batch(lps, opts=oo, threads=oracle_threads())


def compare(batch, gpu, ref, idx=None, rtol=RTOL):
    """Assert parity of GPU results (full batch layout) against oracle results
    for LPs ``idx``.  Returns counts: LPs compared and LPs whose obj, x and y
    are bitwise equal."""
    idx = np.arange(batch.num_lps) if idx is None else np.asarray(idx)
    x_off = batch.x_offsets()
    y_off = batch.y_offsets()
    bitwise = 0
    for t, k in enumerate(idx):
        k = int(k)
        m, n = int(batch.m[k]), int(batch.n[k])
        gs, rs = int(gpu["status"][k]), int(ref["status"][t])
        assert gs == rs, f"LP {k}: status gpu {gs} oracle {rs}"
        gi, ri = int(gpu["iters"][k]), int(ref["iters"][t])
        assert gi == ri, f"LP {k}: iterations gpu {gi} oracle {ri}"
        go, ro = float(gpu["obj"][k]), float(ref["obj"][t])
        assert abs(go - ro) <= rtol * max(1.0, abs(ro)), f"LP {k}: obj gpu {go!r} oracle {ro!r}"
        gx = gpu["x"][x_off[k]:x_off[k] + n]
        rx = ref["x"][t]
        np.testing.assert_allclose(gx, rx, rtol=rtol, atol=rtol * max(1.0, float(np.abs(rx).max(initial=0))),
                                   err_msg=f"LP {k}: x")
        gy = gpu["y"][y_off[k]:y_off[k] + m]
        ry = ref["y"][t]
        np.testing.assert_allclose(gy, ry, rtol=rtol, atol=rtol * max(1.0, float(np.abs(ry).max(initial=0))),
                                   err_msg=f"LP {k}: y")
        bitwise += int(go == ro and np.array_equal(gx, rx) and np.array_equal(gy, ry))
    return len(idx), bitwise
