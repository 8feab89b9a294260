"""GPU parity: the CUDA solver (through the C ABI) against the CPU oracle,
element by element, on seeded inputs shaped like the benchmark workloads,
plus edge cases.  Status and pivot counts must match exactly; objective, x
and y within 1e-10 relative (both sides run the same FP64 operations in the
same order, so they are expected to be bitwise equal)."""
import json
import glob
import os

import numpy as np
import pytest

from paper_1802_08557_gb300 import lpbatch as lpb
from paper_1802_08557_gb300 import workloads as W
import oracle
from parity_util import compare, gpu_solve, oracle_solve

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1802_08557_gb300 import build
    build.build()
    lpb.load()


def _check(batch, **kw):
    g = gpu_solve(batch, **{k: v for k, v in kw.items() if k in ("device_data", "opts")})
    r = oracle_solve(batch, opts=kw.get("opts"))
    n, bitwise = compare(batch, g, r)
    return g, r, n, bitwise


def test_golden_examples_through_abi():
    cases = [json.load(open(p)) for p in sorted(glob.glob(os.path.join(GOLDEN, "worked_*.json")))]
    batch = W.pack("golden", [(np.array(g["A"], float), np.array(g["b"], float), np.array(g["c"], float))
                              for g in cases])
    g = gpu_solve(batch)
    xo, yo = batch.x_offsets(), batch.y_offsets()
    for k, case in enumerate(cases):
        m, n = len(case["b"]), len(case["c"])
        assert g["status"][k] == case["status"], case["name"]
        assert g["iters"][k] == case["iters"], case["name"]
        assert g["obj"][k] == case["obj"], case["name"]
        np.testing.assert_array_equal(g["x"][xo[k]:xo[k] + n], case["x"])
        np.testing.assert_array_equal(g["y"][yo[k]:yo[k] + m], case["y"])


def test_tiny_ragged_batch_matches_oracle():
    from test_oracle_pins import tiny_lps
    batch = W.pack("tiny", tiny_lps(2024, 900))
    g, r, n, bitwise = _check(batch)
    assert set(np.unique(g["status"])) >= {0, 1, 2}
    assert g["plan"]["num_groups"] >= 1
    assert bitwise == n


def test_dense5x5_full_workload():
    batch = W.WORKLOADS["dense5x5_1k"]()
    g, r, n, bitwise = _check(batch)
    assert np.all(g["status"] == lpb.LP_OPTIMAL)
    assert bitwise == n


def test_dense50x50_phase1_several_tiles():
    batch = W.mixed_sign_dense(3000, 50, 50, start=500)
    g, r, n, bitwise = _check(batch)
    assert set(np.unique(g["status"])) == {0, 1, 2}
    assert np.all(g["status"][batch.kind == W.KIND_INFEASIBLE] == lpb.LP_INFEASIBLE)
    assert np.all(g["status"][batch.kind == W.KIND_UNBOUNDED] == lpb.LP_UNBOUNDED)
    assert g["plan"]["num_phase1"] > 0
    assert bitwise == n


def test_support_function_subset():
    batch = W.support_function(2000, start=7)
    g, r, n, bitwise = _check(batch)
    assert bitwise == n


def test_shared_matrix_200x100_and_phase1_at_size():
    batch = W.shared_matrix_family(24, m=200, n=100)
    # force a phase I on some of them at the full 200 x 100 size
    B = batch.b.reshape(24, 200)
    B[::3, ::17] *= -0.05
    g, r, n, bitwise = _check(batch)
    assert g["plan"]["num_phase1"] >= 8
    assert bitwise == n


def test_uneven_sizes_resident_range():
    batch = W.uneven_dense(150, lo=10, hi=500, max_elems=20000)
    g, r, n, bitwise = _check(batch)
    assert g["plan"]["num_groups"] > 3
    assert bitwise == n


def test_edge_shapes():
    rng = np.random.default_rng(5)
    lps = []
    lps.append((np.array([[2.0]]), np.array([3.0]), np.array([1.0])))          # 1 x 1
    lps.append((np.array([[-1.0]]), np.array([-2.0]), np.array([-1.0])))       # 1 x 1, phase I
    lps.append((np.zeros((3, 2)), np.array([1.0, 0.0, 2.0]), np.array([-1.0, -2.0])))  # zero A
    lps.append((np.zeros((2, 2)), np.array([1.0, 1.0]), np.array([1.0, 0.0])))  # zero A, unbounded
    # every b_i < 0 (k = m): -A x <= -b with A, b > 0, c < 0 (bounded)
    lps.append((-rng.uniform(0.5, 1, (6, 6)), -rng.uniform(0.5, 1, 6), -rng.uniform(0.1, 1, 6)))
    lps.append((rng.uniform(-1, 1, (1, 40)), np.array([-0.5]), rng.uniform(-1, 1, 40)))   # m = 1 wide
    lps.append((rng.uniform(-1, 1, (60, 1)), rng.uniform(-1, 2, 60), np.array([0.7])))    # n = 1 tall
    lps.append((np.ones((4, 4)), np.zeros(4), np.ones(4)))                                # fully degenerate
    batch = W.pack("edges", lps)
    g, r, n, bitwise = _check(batch)
    assert bitwise == n


def test_iteration_limit_parity():
    batch = W.mixed_sign_dense(300, 30, 30, start=11)
    opts = lpb.lpb_default_opts(max_iters=7)
    g, r, n, bitwise = _check(batch, opts=opts)
    assert np.sum(g["status"] == lpb.LP_ITER_LIMIT) > 100
    assert bitwise == n


def test_thread_count_does_not_change_results():
    batch = W.mixed_sign_dense(400, 40, 40, start=99)
    base = gpu_solve(batch)
    for t in (32, 64, 256, 512):
        g = gpu_solve(batch, opts=lpb.lpb_default_opts(block_threads=t))
        for key in ("status", "iters", "obj", "x", "y"):
            np.testing.assert_array_equal(g[key], base[key], err_msg=f"threads={t} {key}")


def test_host_and_device_inputs_agree_and_resolve_is_deterministic():
    batch = W.mixed_sign_dense(500, 25, 35, start=3)
    a = gpu_solve(batch, device_data=True)
    b = gpu_solve(batch, device_data=False)
    s = lpb.BatchSolver(batch)
    s.solve(); c1 = s.results()
    s.solve(); c2 = s.results()
    s.close()
    for key in ("status", "iters", "obj", "x", "y"):
        np.testing.assert_array_equal(a[key], b[key])
        np.testing.assert_array_equal(c1[key], c2[key])
        np.testing.assert_array_equal(a[key], c1[key])


def test_errors_are_codes():
    bad = W.pack("nan", [(np.array([[np.nan]]), np.array([1.0]), np.array([1.0]))])
    for device_data in (True, False):
        with pytest.raises(lpb.LPBError) as ei:
            lpb.BatchSolver(bad, device_data=device_data)
        assert ei.value.code == lpb.LPB_EINVAL and "non-finite" in str(ei.value)
    s = lpb.BatchSolver(W.positive_dense(2, 3, 3))
    with pytest.raises(lpb.LPBError) as ei:
        lpb.lp_batch_results(s.h, np.zeros(2, np.int32))
    assert ei.value.code == lpb.LPB_ENOTSOLVED
    s.close()


@pytest.mark.slow
def test_full_size_dense50x50_100k_sampled():
    """The benchmark workload at full size in the benchmark's launch
    configuration: 1e5 LPs of 50 x 50.  A seeded sample is compared with the
    oracle element by element; every LP is checked for properties that hold at
    any size."""
    batch = W.WORKLOADS["dense50x50_phase1_100k"]()
    g = gpu_solve(batch)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(batch.num_lps, 600, replace=False))
    idx = np.concatenate([idx, [0, batch.num_lps - 1]])
    r = oracle_solve(batch, idx)
    n, bitwise = compare(batch, g, r, idx)
    assert bitwise == n
    st = g["status"]
    assert np.all(np.isin(st, [0, 1, 2]))
    assert np.all(st[batch.kind == W.KIND_INFEASIBLE] == lpb.LP_INFEASIBLE)
    assert np.all(st[batch.kind == W.KIND_UNBOUNDED] == lpb.LP_UNBOUNDED)
    # primal feasibility of every optimal LP
    A = batch.A.reshape(-1, 50, 50)
    b = batch.b.reshape(-1, 50)
    c = batch.c.reshape(-1, 50)
    x = g["x"].reshape(-1, 50)
    opt = st == lpb.LP_OPTIMAL
    viol = np.einsum("kij,kj->ki", A[opt], x[opt]) - b[opt]
    assert viol.max() <= 1e-8
    assert x[opt].min() >= -1e-9
    # objective equals c^T x
    np.testing.assert_allclose(np.einsum("kj,kj->k", c[opt], x[opt]), g["obj"][opt], rtol=1e-9, atol=1e-9)


def test_screen_rare_paths_extreme_magnitudes():
    """Rows whose right-hand side or pivot-column entry lies outside
    [2^-100, 2^100] skip the FP32 ratio screen; LPs with exactly equal
    reduced costs / ratios take the exact FP64 tie path."""
    rng = np.random.default_rng(77)
    lps = []
    for t in range(120):
        m, n = int(rng.integers(2, 20)), int(rng.integers(2, 20))
        A = rng.uniform(-1, 1, (m, n))
        b = rng.uniform(-0.5, 2, m)
        c = rng.uniform(-1, 1, n)
        s = [1e35, 1e-35, 1e200, 1e-200][t % 4]
        if t % 3 == 0:
            b = b * s
        elif t % 3 == 1:
            A = A * s
        else:
            A = np.round(A * 3)
            b = np.round(b * 3)
            c = np.round(c * 3)
        lps.append((A, b, c))
    batch = W.pack("extreme", lps)
    g, r, n, bitwise = _check(batch)
    assert bitwise == n


@pytest.mark.parametrize("tau", [0.0, 1e-9, 1e-3])
def test_tie_window_settings(tau):
    from test_oracle_pins import tiny_lps
    lps = tiny_lps(31, 300) + [W.mixed_sign_dense(200, 20, 20, start=5).lp(k) for k in range(200)]
    batch = W.pack("tau", lps)
    g, r, n, bitwise = _check(batch, opts=lpb.lpb_default_opts(tau=tau))
    assert bitwise == n


@pytest.mark.parametrize("tau", [0.0, 1e-3])
def test_streamed_staged_update_extreme_values_and_ties(tau):
    """The streamed kernel (staged update, shared-memory pivot column) on LPs
    that take its rare paths: right-hand sides and entries outside [2^-100,
    2^100] (unscreened rows), integer data with exact ties in Steps 1 and 2,
    degenerate and phase-I LPs, infeasible and unbounded ones -- with and
    without a tie window -- against the oracle bit for bit."""
    rng = np.random.default_rng(131)
    lps = []
    for t in range(24):
        m, n = int(rng.integers(20, 70)), int(rng.integers(20, 70))
        A = rng.uniform(-1, 1, (m, n))
        b = rng.uniform(-0.5, 2, m)
        c = rng.uniform(-1, 1, n)
        kind = t % 4
        if kind == 0:
            b = b * [1e35, 1e-35, 1e200, 1e-200][(t // 4) % 4]
        elif kind == 1:
            A = A * [1e35, 1e-35, 1e120, 1e-120][(t // 4) % 4]
        elif kind == 2:
            A, b, c = np.round(A * 3), np.round(b * 3), np.round(c * 3)  # exact ties
        else:
            b[: m // 2] = 0.0  # degenerate
        lps.append((A, b, c))
    batch = W.pack("streamed_extreme", lps)
    g, r, n, bitwise = _check(batch, opts=lpb.lpb_default_opts(tau=tau, schedule=lpb.LPB_SCHED_STREAMED))
    assert g["plan"]["num_streamed"] == batch.num_lps
    assert len(set(r["status"].tolist())) >= 3  # optimal, infeasible and unbounded among them
    assert bitwise == n


def test_streamed_kernel_matches_resident_bitwise():
    """The same LPs through the global-workspace kernel and the shared-memory
    kernel give identical results (same per-LP code, different storage)."""
    batch = W.mixed_sign_dense(600, 50, 50, start=1234)
    a = gpu_solve(batch)
    b = gpu_solve(batch, opts=lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_STREAMED))
    assert b["plan"]["num_streamed"] == batch.num_lps and b["plan"]["workspace_bytes"] > 0
    assert a["plan"]["num_streamed"] == 0
    for key in ("status", "iters", "obj", "x", "y"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.parametrize("schedule", ["auto", "streamed", "cluster"])
def test_large_lps_take_the_cluster_or_streamed_path(schedule):
    """Tableaux above one CTA's shared memory (e.g. 500 x 500) are solved in a
    global workspace (AUTO: those LPs only; STREAMED: every LP) or split over a
    thread-block cluster's shared memory (CLUSTER); compared with the oracle
    bit for bit, phase I included."""
    rng = np.random.default_rng(8)
    lps = []
    for m, n in [(500, 500), (320, 260), (180, 420), (260, 200), (400, 90)]:
        A = rng.uniform(0, 1, (m, n))
        b = rng.uniform(1, 100, m)
        c = rng.uniform(0, 1, n)
        lps.append((A, b, c))
    A = rng.uniform(0, 1, (250, 150)); b = rng.uniform(1, 100, 250); b[::25] *= -0.01
    lps.append((A, b, rng.uniform(0, 1, 150)))                         # phase I, streamed
    lps.append((rng.uniform(-1, 1, (300, 300)), rng.uniform(-5, 10, 300), rng.uniform(-1, 1, 300)))
    lps += [W.mixed_sign_dense(30, 40, 40, start=9).lp(k) for k in range(30)]  # resident ones alongside
    batch = W.pack("large", lps)
    sched = {"auto": lpb.LPB_SCHED_AUTO, "streamed": lpb.LPB_SCHED_STREAMED, "cluster": lpb.LPB_SCHED_CLUSTER}
    g, r, n, bitwise = _check(batch, opts=lpb.lpb_default_opts(schedule=sched[schedule]))
    if schedule == "cluster":
        assert g["plan"]["num_cluster"] == 7 and g["plan"]["num_streamed"] == 0
        assert g["plan"]["num_resident"] == 30
    elif schedule == "auto":
        assert g["plan"]["num_streamed"] == 7 and g["plan"]["num_cluster"] == 0
        assert g["plan"]["num_resident"] == 30
    else:
        assert g["plan"]["num_streamed"] == batch.num_lps
    assert bitwise == n


def test_streamed_tableaux_beyond_the_staging_buffer():
    """The streamed kernel stages its update through shared memory when the
    LP's pivot row and column fit beside the rings (R + LD up to ~2,000
    doubles), else it runs the plain loop: an LP on each side of that limit
    (one with phase I and a retired artificial column), and tall and wide
    shapes whose chunks end mid-row, against the oracle bit for bit."""
    rng = np.random.default_rng(21)
    lps = []
    A = rng.uniform(0, 1, (400, 1700)); lps.append((A, rng.uniform(1, 100, 400), rng.uniform(0, 1, 1700)))  # plain
    A = rng.uniform(0, 1, (300, 1300)); b = rng.uniform(1, 100, 300); b[::37] *= -0.01
    lps.append((A, b, rng.uniform(0, 1, 1300)))                                     # staged, phase I
    A = rng.uniform(0, 1, (900, 130)); lps.append((A, rng.uniform(1, 100, 900), rng.uniform(0, 1, 130)))
    A = rng.uniform(0, 1, (140, 257)); lps.append((A, rng.uniform(1, 100, 140), rng.uniform(0, 1, 257)))
    batch = W.pack("staging", lps)
    g, r, n, bitwise = _check(batch, opts=lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_STREAMED))
    assert g["plan"]["num_streamed"] == batch.num_lps
    assert bitwise == n
    assert int(g["status"][0]) == 0 and int(g["iters"][0]) > 0


def test_cluster_kernel_matches_streamed_bitwise():
    """Mixed-sign 260 x 260 LPs (phase I, infeasible and unbounded ones among
    them) on thread-block clusters and in the global workspace: identical."""
    batch = W.mixed_sign_dense(24, 260, 260, start=4321)
    a = gpu_solve(batch, opts=lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_CLUSTER))
    b = gpu_solve(batch, opts=lpb.lpb_default_opts(schedule=lpb.LPB_SCHED_STREAMED))
    assert a["plan"]["num_cluster"] == batch.num_lps and b["plan"]["num_cluster"] == 0
    assert len(set(a["status"].tolist())) >= 2
    for key in ("status", "iters", "obj", "x", "y"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_solve_host_equals_create_solve_results(prec):
    """lp_solve_host (host buffers in, host results out, the batch split into
    chunks whose input copies overlap the previous chunk's solve) gives every
    LP's results bit for bit as one create + solve + results of the whole
    batch, for several chunk counts, pinned and pageable inputs, and a batch
    whose LPs share one A (repeated offsets)."""
    import torch
    opts = lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64 if prec == "fp64" else lpb.LP_PREC_FP32_REFINE)
    for batch in (W.mixed_sign_dense(3001, 30, 20, start=123), W.support_function(2000, start=7)):
        ref = gpu_solve(batch, opts=opts)
        N = batch.num_lps
        for chunks, pinned in ((0, True), (1, False), (3, True), (7, False)):
            if pinned:
                A, b, c = (torch.from_numpy(getattr(batch, k)).pin_memory() for k in ("A", "b", "c"))
            else:
                A, b, c = batch.A, batch.b, batch.c
            st, it = np.zeros(N, np.int32), np.zeros(N, np.int32)
            ob = np.zeros(N)
            x = np.zeros(int(batch.n.astype(np.int64).sum()))
            y = np.zeros(int(batch.m.astype(np.int64).sum()))
            lpb.lp_solve_host(batch.m, batch.n, batch.a_off, A, batch.b_off, b, batch.c_off, c, st, it, ob, x, y,
                              opts=opts, chunks=chunks)
            for key, v in (("status", st), ("iters", it), ("obj", ob), ("x", x), ("y", y)):
                np.testing.assert_array_equal(v, ref[key], err_msg=f"{key} chunks={chunks}")


def test_solve_host_reports_errors_of_a_later_chunk():
    """A non-finite entry in the last chunk: lp_solve_host returns LPB_EINVAL
    (the chunks' input checks are read after their solves; the check zeroes
    the entry in the device copy, so the solve runs on finite data), writes no
    results, releases everything, and a later call on good data still works."""
    batch = W.mixed_sign_dense(400, 10, 8, start=5)
    A = batch.A.copy()
    A[-1] = np.inf
    N = batch.num_lps
    st, it, ob = np.zeros(N, np.int32), np.zeros(N, np.int32), np.zeros(N)
    x = np.zeros(int(batch.n.astype(np.int64).sum()))
    with pytest.raises(lpb.LPBError) as e:
        lpb.lp_solve_host(batch.m, batch.n, batch.a_off, A, batch.b_off, batch.b, batch.c_off, batch.c,
                          st, it, ob, x, chunks=4)
    assert e.value.code == lpb.LPB_EINVAL
    assert "non-finite" in str(e.value)
    assert not st.any() and not it.any() and not ob.any() and not x.any()
    lpb.lp_solve_host(batch.m, batch.n, batch.a_off, batch.A, batch.b_off, batch.b, batch.c_off, batch.c,
                      st, it, ob, x, chunks=4)
    ref = gpu_solve(batch)
    np.testing.assert_array_equal(ob, ref["obj"])


def test_solve_host_non_finite_rhs_in_a_middle_chunk():
    """b_i = -inf counts as a phase-I row in the host's plan, while the
    device copy the solve reads holds 0 (the check zeroes it): the solve needs
    no more shared memory than planned, and the call returns LPB_EINVAL with
    no results written.  NaN in c: the same.  Then a good call still works."""
    batch = W.mixed_sign_dense(600, 12, 9, start=40)
    N = batch.num_lps
    st, it, ob = np.zeros(N, np.int32), np.zeros(N, np.int32), np.zeros(N)
    x = np.zeros(int(batch.n.astype(np.int64).sum()))
    for which in ("b", "c"):
        b, c = batch.b.copy(), batch.c.copy()
        if which == "b":
            b[int(batch.b_off[300]) + 3] = -np.inf
        else:
            c[int(batch.c_off[301]) + 1] = np.nan
        with pytest.raises(lpb.LPBError) as e:
            lpb.lp_solve_host(batch.m, batch.n, batch.a_off, batch.A, batch.b_off, b, batch.c_off, c,
                              st, it, ob, x, chunks=3)
        assert e.value.code == lpb.LPB_EINVAL and "non-finite" in str(e.value)
        assert not st.any() and not ob.any() and not x.any()
    lpb.lp_solve_host(batch.m, batch.n, batch.a_off, batch.A, batch.b_off, batch.b, batch.c_off, batch.c,
                      st, it, ob, x, chunks=3)
    np.testing.assert_array_equal(ob, gpu_solve(batch)["obj"])
