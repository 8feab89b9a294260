"""GPU: FP32 tableau + FP64 certificate (LP_PREC_FP32_REFINE) against the
FP64 oracle.  Status must equal the oracle's exactly; optimal objectives must
agree within 1e-9 relative (the mixed path's accuracy target); every optimum
returned must pass an FP64 duality certificate computed here in numpy."""
import numpy as np
import pytest

from paper_1802_08557_gb300 import lpbatch as lpb
from paper_1802_08557_gb300 import workloads as W
from parity_util import gpu_solve, oracle_solve

pytestmark = pytest.mark.gpu

OBJ_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1802_08557_gb300 import build
    build.build()
    lpb.load()


def mixed_opts(**kw):
    return lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE, **kw)


def check_mixed(batch, max_fallback_frac=1.0, cert_mask=None):
    g = gpu_solve(batch, opts=mixed_opts())
    r = oracle_solve(batch)
    xo, yo = batch.x_offsets(), batch.y_offsets()
    for k in range(batch.num_lps):
        assert g["status"][k] == r["status"][k], f"LP {k}: status {g['status'][k]} vs oracle {r['status'][k]}"
        if r["status"][k] == 1:
            # infeasible: y is a Farkas certificate (y >= 0, A^T y >= 0, b^T y < 0)
            A, b, c = batch.lp(k)
            y = g["y"][yo[k]:yo[k] + A.shape[0]]
            # (tolerances as in the oracle's own certificate pins)
            scale = max(1.0, np.abs(A).max(), np.abs(b).max(), np.abs(c).max())
            ys = max(1.0, float(np.abs(y).max()))
            assert y.min() >= -1e-7 * ys, f"LP {k}: Farkas y has negative entries"
            assert np.all(A.T @ y >= -1e-7 * scale * ys), f"LP {k}: A^T y < 0"
            assert float(b @ y) < 0.0, f"LP {k}: b^T y >= 0"
        if r["status"][k] != 0:
            continue
        A, b, c = batch.lp(k)
        m, n = A.shape
        go, ro = g["obj"][k], r["obj"][k]
        assert abs(go - ro) <= OBJ_RTOL * max(1.0, abs(ro)), f"LP {k}: obj {go!r} vs {ro!r}"
        if cert_mask is not None and not cert_mask[k]:
            continue
        x = g["x"][xo[k]:xo[k] + n]
        y = g["y"][yo[k]:yo[k] + m]
        sb = max(1.0, np.abs(b).max())
        sc = max(1.0, np.abs(c).max())
        assert x.min() >= -1e-9 * sb
        assert np.all(A @ x <= b + 1e-9 * sb + 1e-12 * (np.abs(A) @ np.abs(x)))
        assert y.min() >= -1e-9 * sc
        assert np.all(A.T @ y >= c - 1e-9 * sc - 1e-12 * (np.abs(A).T @ np.abs(y)))
        assert abs(float(c @ x) - float(b @ y)) <= 1e-9 * max(1.0, abs(float(c @ x)))
    plan = g["plan"]
    assert plan["internal_errors"] == 0, plan
    assert plan["num_mixed"] > 0
    assert plan["num_fallback"] <= max_fallback_frac * plan["num_mixed"], plan
    return g, r


def test_mixed_dense50x50_phase1():
    batch = W.mixed_sign_dense(3000, 50, 50, start=777)
    # about 1.2% are re-solved in FP64 (ill-conditioned bases, phase-I
    # degeneracy); a certificate that stopped converging would exceed 5%
    g, r = check_mixed(batch, max_fallback_frac=0.05)
    assert set(np.unique(g["status"])) == {0, 1, 2}


def test_mixed_dense5x5():
    check_mixed(W.WORKLOADS["dense5x5_1k"](), max_fallback_frac=0.05)


def test_mixed_support_function():
    check_mixed(W.support_function(2000, start=3), max_fallback_frac=0.05)


def test_mixed_shared_matrix_family():
    check_mixed(W.shared_matrix_family(40, m=200, n=100), max_fallback_frac=0.25)


def test_mixed_tiny_and_degenerate():
    from test_oracle_pins import tiny_lps
    check_mixed(W.pack("tiny", tiny_lps(4242, 600)))


def test_mixed_extreme_scales_fall_back_correctly():
    """LPs with data outside [2^-60, 2^60] go straight to the FP64 kernel
    (their results are the FP64 simplex's: status and objective checked);
    1e6-scaled ones stay on the mixed path and must be certified."""
    rng = np.random.default_rng(9)
    lps = []
    scales = []
    for t in range(60):
        m, n = int(rng.integers(3, 15)), int(rng.integers(3, 15))
        s = [1e30, 1e-30, 1e6][t % 3]
        scales.append(s)
        lps.append((rng.uniform(-1, 1, (m, n)) * s, rng.uniform(-0.5, 2, m), rng.uniform(-1, 1, n)))
    in_range = np.array([s == 1e6 for s in scales])
    g, r = check_mixed(W.pack("scales", lps), cert_mask=in_range)
    assert g["plan"]["num_fallback"] >= int((~in_range).sum())


def test_mixed_uneven_shapes_against_oracle():
    """The uneven workload's shapes (m, n log-uniform in [10, 500]): its 60
    largest LPs of the first 1500 (FP32 tableaux above one CTA's shared
    memory: the streamed mixed kernel, with FP64 re-solves on thread-block
    clusters or streamed) and 90 evenly spaced others (shared-memory kernels),
    in one batch.  Status equal to the oracle's, objective within 1e-9, and
    every optimum certified in numpy."""
    full = W.uneven_dense(1500, start=0)
    size = full.m.astype(np.int64) * full.n.astype(np.int64)
    big = np.argsort(-size, kind="stable")[:60]
    rest = np.setdiff1d(np.arange(full.num_lps), big)[::15][:90]
    batch = full.subset(np.sort(np.concatenate([big, rest])))
    g, r = check_mixed(batch)
    s = lpb.BatchSolver(batch, opts=mixed_opts())
    try:
        kinds = {gr["kind"] for gr in lpb.lp_batch_groups(s.h)}
    finally:
        s.close()
    assert 4 in kinds and 0 in kinds, kinds  # both the streamed and the shared-memory mixed kernels ran
    assert int(np.sum(r["status"] == 0)) == batch.num_lps  # positive data: all optimal


def test_mixed_streamed_matches_shared_memory_bitwise():
    """LPB_SCHED_STREAMED with FP32_REFINE puts every LP's FP32 tableau in a
    global workspace slot (persistent 512-thread CTAs, group kind 4).  The
    per-LP arithmetic does not depend on where the tableau lives or on the
    thread count, so every output equals the shared-memory kernels' bit for
    bit (the uneven batch includes m >= 64, where certificate sums are split)."""
    for batch in (W.mixed_sign_dense(1500, 50, 50, start=99), W.uneven_dense(300, lo=8, hi=150, start=17)):
        a = gpu_solve(batch, opts=mixed_opts())
        s = lpb.BatchSolver(batch, opts=mixed_opts(schedule=lpb.LPB_SCHED_STREAMED))
        try:
            s.solve()
            b = s.results()
            plan = s.plan_info()
            kinds = {g["kind"] for g in lpb.lp_batch_groups(s.h)}
        finally:
            s.close()
        assert plan["internal_errors"] == 0, plan
        assert plan["num_streamed"] == batch.num_lps and plan["num_resident"] == 0, plan
        assert kinds == {4}, kinds
        assert plan["num_fallback"] == a["plan"]["num_fallback"]
        for key in ("status", "iters", "obj", "x", "y"):
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_mixed_large_lps_and_their_fp64_streamed_re_solve():
    """FP32 tableaux above one CTA's shared memory run in the streamed mixed
    kernel; LPs whose FP64 tableau exceeds one CTA and that the mixed path does
    not certify (here: an entry outside the FP32 range) are re-solved by the
    FP64 cluster kernel, whose answer equals the FP64 path's bit for bit.
    Feasible and infeasible phase-I LPs are among them.  Every status equals
    the FP64 path's, every optimal objective agrees within 1e-9."""
    rng = np.random.default_rng(5)
    lps, forced = [], []
    for t in range(8):
        # t < 4: FP32 tableau fits one CTA, FP64 does not; t >= 4: neither fits
        m, n = (170 + 10 * t, 160 + 5 * t) if t < 4 else (250 + 10 * t, 240 + 10 * t)
        A = rng.uniform(0.0, 1.0, (m, n))
        b = rng.uniform(1.0, 100.0, m)
        c = rng.uniform(0.0, 1.0, n)
        if t in (2, 3, 6, 7):
            # rows with b_i < 0 (phase I): feasible when those rows of A are
            # negated too (t = 2, 6), infeasible with A >= 0 (t = 3, 7)
            b[::7] = -rng.uniform(0.001, 0.01, b[::7].shape)
            if t in (2, 6):
                A[::7] = -A[::7]
        if t % 2 == 1:
            A[0, 0] = 2.0 ** 61  # above the FP32 pass's 2^60 bound: straight to the FP64 re-solve
        forced.append(t % 2 == 1)
        lps.append((A, b, c))
    batch = W.pack("large_mixed", lps)
    g = gpu_solve(batch, opts=mixed_opts())
    f = gpu_solve(batch, opts=lpb.lpb_default_opts())
    s = lpb.BatchSolver(batch, opts=mixed_opts())
    try:
        kinds = sorted({gg["kind"] for gg in lpb.lp_batch_groups(s.h)})
    finally:
        s.close()
    assert kinds == [0, 4], kinds
    assert g["plan"]["num_fallback"] >= sum(forced)
    np.testing.assert_array_equal(g["status"], f["status"])
    assert set(f["status"][[3, 7]]) == {1} and f["status"][2] == 0 and f["status"][6] == 0
    opt = f["status"] == 0
    assert opt.any()
    np.testing.assert_allclose(g["obj"][opt], f["obj"][opt], rtol=OBJ_RTOL, atol=OBJ_RTOL)
    xo, yo = batch.x_offsets(), batch.y_offsets()
    for k in np.nonzero(forced)[0]:
        m, n = int(batch.m[k]), int(batch.n[k])
        assert g["iters"][k] == f["iters"][k] and g["obj"][k] == f["obj"][k]
        np.testing.assert_array_equal(g["x"][xo[k]:xo[k] + n], f["x"][xo[k]:xo[k] + n])
        np.testing.assert_array_equal(g["y"][yo[k]:yo[k] + m], f["y"][yo[k]:yo[k] + m])


@pytest.mark.slow
def test_full_size_repeat_solves_are_identical():
    """1e5 LPs of 50 x 50: solving twice gives bitwise identical results on
    both paths, and no kernel reports an internal-consistency failure."""
    batch = W.WORKLOADS["dense50x50_phase1_100k"]()
    for opts in (lpb.lpb_default_opts(), mixed_opts()):
        s = lpb.BatchSolver(batch, opts=opts)
        try:
            s.solve()
            r1 = s.results()
            p1 = s.plan_info()
            s.solve()
            r2 = s.results()
            p2 = s.plan_info()
        finally:
            s.close()
        assert p1["internal_errors"] == 0 and p2["internal_errors"] == 0, (p1, p2)
        assert p1["num_fallback"] == p2["num_fallback"]
        for key in ("status", "iters", "obj", "x", "y"):
            np.testing.assert_array_equal(r1[key], r2[key], err_msg=key)


@pytest.mark.parametrize("threads", [32, 128])
def test_mixed_warp_and_block_variants(threads):
    """The FP32 stage runs one warp per LP for small tableaux and one CTA per
    LP for larger ones; both must certify the same answers as the oracle."""
    batch = W.mixed_sign_dense(800, 50, 50, start=31337)
    g = gpu_solve(batch, opts=mixed_opts(block_threads=threads))
    r = oracle_solve(batch)
    np.testing.assert_array_equal(g["status"], r["status"])
    opt = r["status"] == 0
    np.testing.assert_allclose(g["obj"][opt], r["obj"][opt], rtol=OBJ_RTOL, atol=OBJ_RTOL)
    big = W.shared_matrix_family(12, m=200, n=100, start=5)
    g = gpu_solve(big, opts=mixed_opts(block_threads=threads))
    r = oracle_solve(big)
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_allclose(g["obj"], r["obj"], rtol=OBJ_RTOL, atol=OBJ_RTOL)


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
def test_repeat_solves_identical_per_group_size(threads):
    """Every thread-group size gives the same bits on a repeat solve (the
    phase-I LPs exercise the artificial-column retirement and the ranking of
    negative rows, both of which order shared-memory accesses across warps)."""
    batch = W.mixed_sign_dense(20000, 50, 50, start=777)
    s = lpb.BatchSolver(batch, opts=mixed_opts(block_threads=threads))
    try:
        s.solve()
        r1, p1 = s.results(), s.plan_info()
        s.solve()
        r2, p2 = s.results(), s.plan_info()
    finally:
        s.close()
    assert p1["internal_errors"] == 0 and p2["internal_errors"] == 0
    assert p1["num_fallback"] == p2["num_fallback"]
    for key in ("status", "iters", "obj", "x", "y"):
        np.testing.assert_array_equal(r1[key], r2[key], err_msg=key)


def test_stage_timing_reports_both_stages():
    """lp_batch_set_timing / lp_batch_stage_times: CUDA-event times of the
    launch groups and of the FP64 re-solve, averaged over the solves since
    timing was enabled; an error when timing is off."""
    batch = W.mixed_sign_dense(400, 50, 50, start=99)
    s = lpb.BatchSolver(batch, opts=mixed_opts())
    try:
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_stage_times(s.h)
        lpb.lp_batch_set_timing(s.h, True)
        s.solve()
        s.solve()
        main_ms, fb_ms, n = lpb.lp_batch_stage_times(s.h)
        assert n == 2 and main_ms > 0.0 and fb_ms >= 0.0
        assert lpb.lp_batch_stage_times(s.h)[2] == 0  # read resets the count
        lpb.lp_batch_set_timing(s.h, False)
        s.solve()
        assert s.plan_info()["internal_errors"] == 0
    finally:
        s.close()
