"""Launch forms of uneven batches: one CTA per LP or persistent CTAs over a
work queue (longest work first), thread counts picked by the autotuner, and
the solve captured in a CUDA graph.  None of these may change a single bit of
the results (each LP's arithmetic is the same whatever runs it)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1802_08557_gb300 import lpbatch as lpb
from paper_1802_08557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("status", "iters", "obj", "x", "y")


def _same(a, b):
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _batches():
    return {
        "uneven_fp64": (W.uneven_dense(400, lo=8, hi=120, start=3), lpb.LP_PREC_FP64),
        "dense_mixed": (W.mixed_sign_dense(1500, 30, 30, start=5), lpb.LP_PREC_FP32_REFINE),
        "uneven_mixed": (W.uneven_dense(300, lo=8, hi=90, start=9), lpb.LP_PREC_FP32_REFINE),
    }


@pytest.mark.parametrize("name", ["uneven_fp64", "dense_mixed", "uneven_mixed"])
def test_forced_forms_give_identical_results(name):
    batch, prec = _batches()[name]
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=prec))
    try:
        s.solve()
        ref = s.results()
        groups = lpb.lp_batch_groups(s.h)
        assert groups and sum(g["count"] for g in groups) == batch.num_lps
        for persistent in (True, False):
            for threads in (32, 64, 256):
                for i, g in enumerate(groups):
                    if g["kind"] in (0, 1) and (not persistent or g["smem_bytes"] <= 226 * 1024):
                        lpb.lp_batch_set_group_form(s.h, i, threads, persistent)
                s.solve()
                _same(s.results(), ref)
                assert s.plan_info()["internal_errors"] == 0
                assert all(g["persistent"] == int(persistent) for g in lpb.lp_batch_groups(s.h)
                           if g["kind"] != 2 and g["smem_bytes"] <= 226 * 1024)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["uneven_fp64", "dense_mixed"])
def test_autotune_keeps_results(name):
    batch, prec = _batches()[name]
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=prec))
    try:
        s.solve()
        ref = s.results()
        lpb.lp_batch_autotune(s.h, rounds=1)
        with pytest.raises(lpb.LPBError):
            s.results()  # the trial launches left partial outputs: solve first
        s.solve()
        _same(s.results(), ref)
        tuned = [g for g in lpb.lp_batch_groups(s.h) if g["kind"] != 2]
        assert tuned and all(g["tuned_ms"] >= 0.0 for g in tuned)
    finally:
        s.close()


def test_graph_solve_replays_the_plain_solve():
    batch, prec = _batches()["dense_mixed"]
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=prec))
    try:
        s.solve()
        ref = s.results()
        for _ in range(3):
            lpb.lp_batch_solve_graph(s.h)
            _same(s.results(), ref)
        assert s.plan_info()["num_fallback"] >= 0
        # a changed form drops the graph; the next graph solve recaptures it
        lpb.lp_batch_set_group_form(s.h, 0, 128, True)
        lpb.lp_batch_solve_graph(s.h)
        _same(s.results(), ref)
    finally:
        s.close()


@pytest.mark.parametrize("kind", ["all_one_warp", "none_one_warp"])
def test_mixed_single_launch_warp_mode_bounds(kind):
    """The mixed single launch with every LP in warp mode (small LPs only:
    each CTA switches at its first draw) and with none (every LP above the
    one-warp size): the same bits as the default plan."""
    if kind == "all_one_warp":
        lps = [W.uneven_dense(400, lo=4, hi=40, start=61).lp(k) for k in range(400)]
        lps += [W.mixed_sign_dense(60, 30, 30, start=8).lp(k) for k in range(60)]
    else:
        rng = np.random.default_rng(62)
        lps = [(rng.uniform(0, 1, (m, n)), rng.uniform(1, 100, m), rng.uniform(0, 1, n))
               for m, n in [(130, 90), (100, 120), (160, 70), (95, 95), (140, 140), (300, 250)] * 4]
    batch = W.pack("single_" + kind, lps)
    want = gpu_solve_opts(batch, lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE))
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE,
                                                         schedule=lpb.LPB_SCHED_SINGLE))
    try:
        for _ in range(2):
            s.solve()
            _same(s.results(), want)
            assert s.plan_info()["internal_errors"] == 0
    finally:
        s.close()


def test_lpt_order_and_errors():
    batch = W.uneven_dense(200, lo=8, hi=150, start=11)
    s = lpb.BatchSolver(batch)
    try:
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_set_group_form(s.h, 0, 48, False)   # not a multiple of 32
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_set_group_form(s.h, 10_000, 64, False)
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_autotune(s.h, rounds=0)
    finally:
        s.close()


def gpu_solve_opts(batch, opts):
    s = lpb.BatchSolver(batch, opts=opts)
    try:
        s.solve()
        r = s.results()
        assert s.plan_info()["internal_errors"] == 0
        return r
    finally:
        s.close()


def test_single_launch_schedule_gives_identical_results():
    """LPB_SCHED_SINGLE: the whole uneven batch in one persistent launch (one
    work queue, longest work first; tableaux up to 110 KB in shared memory,
    larger ones in the CTA's global workspace slot) -- the same bits as the
    default plan's many launch groups, large LPs and phase I included, and
    again on a repeat solve and through a graph replay."""
    rng = np.random.default_rng(21)
    lps = [W.uneven_dense(300, lo=8, hi=200, start=40).lp(k) for k in range(300)]
    for m, n in [(300, 250), (420, 160), (260, 300)]:        # tableaux above 110 KB
        lps.append((rng.uniform(0, 1, (m, n)), rng.uniform(1, 100, m), rng.uniform(0, 1, n)))
    A = rng.uniform(-1, 1, (150, 140)); b = rng.uniform(-5, 10, 150); c = rng.uniform(-1, 1, 140)
    lps.append((A, b, c))                                     # phase I, mid size
    lps += [W.mixed_sign_dense(50, 40, 40, start=3).lp(k) for k in range(50)]
    batch = W.pack("single", lps)
    ref = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts())
    try:
        ref.solve()
        want = ref.results()
    finally:
        ref.close()
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_SINGLE))
    try:
        plan = s.plan_info()
        groups = lpb.lp_batch_groups(s.h)
        assert plan["num_groups"] == 1 and len(groups) == 1 and groups[0]["kind"] == 5, groups
        assert groups[0]["count"] == batch.num_lps and plan["num_streamed"] >= 3
        for run in range(2):
            s.solve()
            _same(s.results(), want)
            assert s.plan_info()["internal_errors"] == 0
        lpb.lp_batch_solve_graph(s.h)
        _same(s.results(), want)
    finally:
        s.close()
    # a batch of streamed LPs only: the single launch still gets the shared
    # memory to stage their update, and matches the streamed kernel bit for bit
    big = W.pack("single_big", lps[300:303])
    a = gpu_solve_opts(big, lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_STREAMED))
    b = gpu_solve_opts(big, lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_SINGLE))
    _same(b, a)


def test_mixed_single_launch_gives_identical_results():
    """LPB_SCHED_SINGLE with mixed precision: one persistent launch of the
    mixed per-LP code (each LP's area in shared memory up to 110 KB, else in
    the CTA's global slot), then the FP64 re-solves -- the same bits as the
    default mixed plan, with LPs whose FP32 tableau is resident in one plan and
    streamed in the other, phase I, infeasible and unbounded LPs, and LPs the
    certificate hands to the FP64 re-solve; again on a repeat solve and
    through a graph replay."""
    rng = np.random.default_rng(23)
    lps = [W.uneven_dense(300, lo=8, hi=200, start=41).lp(k) for k in range(300)]
    for m, n in [(300, 250), (180, 170), (200, 190)]:        # FP32 areas above 110 KB
        lps.append((rng.uniform(0, 1, (m, n)), rng.uniform(1, 100, m), rng.uniform(0, 1, n)))
    A = rng.uniform(0, 1, (60, 50)); A[0, 0] = 2.0 ** 61      # above the FP32 pass's 2^60 bound: FP64 re-solve
    lps.append((A, rng.uniform(1, 100, 60), rng.uniform(0, 1, 50)))
    lps += [W.mixed_sign_dense(80, 40, 40, start=5).lp(k) for k in range(80)]
    batch = W.pack("single_mixed", lps)
    opts = lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE)
    ref = lpb.BatchSolver(batch, opts=opts)
    try:
        ref.solve()
        want = ref.results()
        want_plan = ref.plan_info()
    finally:
        ref.close()
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE,
                                                         schedule=lpb.LPB_SCHED_SINGLE))
    try:
        groups = lpb.lp_batch_groups(s.h)
        assert len(groups) == 1 and groups[0]["kind"] == 5 and groups[0]["count"] == batch.num_lps, groups
        for run in range(2):
            s.solve()
            got = s.results()
            _same(got, want)
            plan = s.plan_info()
            assert plan["internal_errors"] == 0 and plan["num_mixed"] == batch.num_lps
            assert plan["num_fallback"] == want_plan["num_fallback"] >= 1
        assert len(set(want["status"].tolist())) == 3
        lpb.lp_batch_solve_graph(s.h)
        _same(s.results(), want)
    finally:
        s.close()
