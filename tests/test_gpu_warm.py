"""Learned warm start on the GPU: the network is trained by the library's own
kernels on LPs the library solved, proposes the active rows of new LPs of the
same family (shared A, varying b and c), and lp_batch_solve_warm certifies the
restricted optimum in FP64 or hands the LP to the cold FP64 solve.

Parity: every status equals the cold FP64 solve's (and the oracle's on a
sample); optimal objectives within 1e-9 relative; certified x primal feasible
and y dual feasible on the full LP; LPs that fall back are bit-identical to the
cold FP64 solve.  Gain: the trained network certifies most LPs, an untrained
one (the method without learning) almost none."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1802_08557_gb300 import lpbatch as lpb
from paper_1802_08557_gb300 import warmstart as WS
from paper_1802_08557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M, N_ = 200, 100


@pytest.fixture(scope="module")
def trained():
    train = W.shared_matrix_family_blocks(100_000)
    net, info = WS.train(train, epochs=3.0, batch_size=1024, seed=0)
    assert info["last_loss"] < 0.2 * info["first_loss"], info
    yield net, train
    net.close()


@pytest.fixture(scope="module")
def test_batch():
    return W.shared_matrix_family(4000, start=0)


def _cold(batch):
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64))
    try:
        s.solve()
        return s.results()
    finally:
        s.close()


def test_warm_solve_matches_cold_and_oracle(trained, test_batch):
    net, _ = trained
    r, plan = WS.solve_warm(test_batch, net, threshold=0.2)
    assert plan["internal_errors"] == 0
    c = _cold(test_batch)
    np.testing.assert_array_equal(r["status"], c["status"])
    opt = c["status"] == 0
    rel = np.abs(r["obj"][opt] - c["obj"][opt]) / np.maximum(1.0, np.abs(c["obj"][opt]))
    assert rel.max() <= 1e-9
    # oracle on a sample
    idx = np.arange(0, test_batch.num_lps, 40)
    ref = oracle.solve_batch([test_batch.lp(int(k)) for k in idx], threads=8)
    np.testing.assert_array_equal(r["status"][idx], ref["status"])
    o = ref["status"] == 0
    assert np.all(np.abs(r["obj"][idx][o] - ref["obj"][o]) <= 1e-9 * np.maximum(1.0, np.abs(ref["obj"][o])))
    # certificates on the full LP from the reported x, y
    xo, yo = test_batch.x_offsets(), test_batch.y_offsets()
    for k in range(0, test_batch.num_lps, 25):
        A, b, cc = test_batch.lp(k)
        x = r["x"][xo[k]:xo[k] + N_]
        y = r["y"][yo[k]:yo[k] + M]
        tol_p = 1e-9 * max(1.0, np.abs(b).max()) * 10
        tol_d = 1e-9 * max(1.0, np.abs(cc).max()) * 10
        assert np.all(A @ x <= b + tol_p) and np.all(x >= -tol_p)
        assert np.all(y >= -tol_d) and np.all(A.T @ y - cc >= -tol_d)
        assert abs(cc @ x - b @ y) <= 1e-9 * max(1.0, abs(cc @ x)) * 10


def test_trained_network_certifies_what_an_untrained_one_cannot(trained, test_batch):
    net, train = trained
    _, plan = WS.solve_warm(test_batch, net, threshold=0.2)
    trained_rate = plan["num_warm_certified"] / test_batch.num_lps
    assert plan["num_warm_certified"] + plan["num_fallback"] == test_batch.num_lps
    untrained = lpb.Mlp(M + N_, 512, 512, M, max_batch=1024, seed=7)
    untrained.fit_scaling(WS.batch_features(train))
    r0, plan0 = WS.solve_warm(test_batch, untrained, threshold=0.2)
    untrained_rate = plan0["num_warm_certified"] / test_batch.num_lps
    untrained.close()
    assert trained_rate >= 0.9, trained_rate
    assert untrained_rate <= 0.1, untrained_rate
    # the untrained run is answered by the cold solve: still correct
    np.testing.assert_array_equal(r0["status"], _cold(test_batch)["status"])


@pytest.mark.parametrize("threshold", [0.2, 0.01])
def test_second_pass_for_rows_beyond_the_first_cap(trained, test_batch, threshold):
    """The first pass holds at most 16 restricted rows; an LP whose rows
    outgrow that (a low threshold proposes more rows) goes to the second pass
    with up to 32, and only then to the cold solve.  Every status equals the
    cold FP64 solve's, optimal objectives within 1e-9; the counts add up."""
    net, _ = trained
    batch = test_batch.subset(np.arange(1500))
    r, plan = WS.solve_warm(batch, net, threshold=threshold)
    assert plan["internal_errors"] == 0
    assert plan["num_warm_certified"] + plan["num_fallback"] == batch.num_lps
    assert 0 <= plan["num_warm_retried"] <= batch.num_lps
    if threshold < 0.1:
        assert plan["num_warm_retried"] > 0, plan  # many proposals above 16 rows
    c = _cold(batch)
    np.testing.assert_array_equal(r["status"], c["status"])
    opt = c["status"] == 0
    rel = np.abs(r["obj"][opt] - c["obj"][opt]) / np.maximum(1.0, np.abs(c["obj"][opt]))
    assert rel.max() <= 1e-9


def test_fallback_lps_are_the_cold_fp64_results(trained, test_batch):
    """With an untrained network nothing is certified: every LP is answered by
    the cold FP64 solve, bit for bit."""
    _, train = trained
    untrained = lpb.Mlp(M + N_, 512, 512, M, max_batch=1024, seed=11)
    untrained.fit_scaling(WS.batch_features(train))
    batch = test_batch.subset(np.arange(1000))
    r, plan = WS.solve_warm(batch, untrained, threshold=0.5)
    untrained.close()
    c = _cold(batch)
    assert plan["num_fallback"] == batch.num_lps - plan["num_warm_certified"]
    if plan["num_warm_certified"] == 0:
        for key in ("status", "iters", "obj", "x", "y"):
            np.testing.assert_array_equal(r[key], c[key], err_msg=key)


def test_constraint_generation_adds_missing_rows(trained, test_batch):
    """A threshold of 0.999 proposes too few rows: the restricted optimum
    violates some, which are added round by round until it is feasible."""
    net, _ = trained
    r, plan = WS.solve_warm(test_batch, net, threshold=0.999)
    c = _cold(test_batch)
    np.testing.assert_array_equal(r["status"], c["status"])
    opt = c["status"] == 0
    assert np.all(np.abs(r["obj"][opt] - c["obj"][opt]) <= 1e-9 * np.maximum(1.0, np.abs(c["obj"][opt])))
    assert plan["num_warm_rounds"] > plan["num_warm_certified"] > 0


def test_features_and_labels(test_batch):
    import torch
    batch = test_batch.subset(np.arange(300))
    s = lpb.BatchSolver(batch, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64))
    try:
        x = torch.empty((300, M + N_), dtype=torch.float32, device="cuda")
        lab = torch.empty((300, M), dtype=torch.float32, device="cuda")
        lpb.lp_batch_features(s.h, x)
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_active_labels(s.h, lab)  # before any solve
        s.solve()
        lpb.lp_batch_active_labels(s.h, lab)
        torch.cuda.synchronize()
        r = s.results()
    finally:
        s.close()
    xs = x.cpu().numpy()
    ys = lab.cpu().numpy()
    for k in range(0, 300, 7):
        A, b, cc = batch.lp(k)
        np.testing.assert_array_equal(xs[k], np.concatenate([b, cc]).astype(np.float32))
        yk = r["y"][k * M:(k + 1) * M]
        np.testing.assert_array_equal(ys[k], ((yk > 0) & (r["status"][k] == 0)).astype(np.float32))


def test_warm_solve_errors(trained):
    net, _ = trained
    uneven = W.uneven_dense(10, lo=5, hi=9)
    s = lpb.BatchSolver(uneven)
    try:
        with pytest.raises(lpb.LPBError) as e:
            lpb.lp_batch_solve_warm(s.h, net, 0.2)
        assert e.value.code == lpb.LPB_EINVAL      # sizes differ
    finally:
        s.close()
    small = W.positive_dense(10, 5, 5)
    s = lpb.BatchSolver(small)
    try:
        with pytest.raises(lpb.LPBError) as e:
            lpb.lp_batch_solve_warm(s.h, net, 0.2)
        assert e.value.code == lpb.LPB_EINVAL      # network widths do not match
        with pytest.raises(lpb.LPBError):
            lpb.lp_batch_solve_warm(s.h, net, 1.5)  # threshold outside (0, 1)
    finally:
        s.close()
