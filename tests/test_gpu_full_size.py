"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (the default plan of each path), on seeded samples the oracle solves
one by one, plus properties checked on every LP:

- 1e5 dense 50 x 50 LPs (about a fifth with phase I), the mixed path of the
  headline: status exact and objective within 1e-9 relative of the oracle on
  602 sampled LPs; on every LP, optimal ones primal feasible with
  c^T x equal to the reported objective and y >= 0 (dual feasible slacks),
  infeasible ones with a Farkas certificate, and the LPs built infeasible or
  unbounded reported so.
- The support function of one polytope (1e5 directions, 40 x 20 after
  x = x+ - x-), both paths: the FP64 path against the oracle element by
  element, the mixed path on status and objective; every LP bounded.
- The uneven batch (2e4 LPs, m and n in [10, 500]), both paths, on an
  evenly spaced sample plus the largest LPs (tableaux in global memory):
  FP64 element by element, mixed on status and objective.

The FP64 paths run the oracle's operations in its order, so they are
expected to agree bit for bit; the mixed path's FP32 pivots may end on
another optimal basis, so x is checked by feasibility, not equality."""
import numpy as np
import pytest

from paper_1802_08557_gb300 import lpbatch as lpb
from paper_1802_08557_gb300 import workloads as W
from parity_util import compare, gpu_solve, oracle_solve

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

OBJ_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1802_08557_gb300 import build
    build.build()
    lpb.load()


def mixed_opts():
    return lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE)


def sample(num, count, seed, extra=()):
    rng = np.random.default_rng(seed)
    idx = rng.choice(num, min(count, num), replace=False)
    return np.unique(np.concatenate([idx, [0, num - 1], np.asarray(extra, dtype=np.int64)])).astype(np.int64)


def check_status_obj(g, r, idx):
    """Status exact, objective within OBJ_RTOL relative on optimal LPs."""
    for t, k in enumerate(idx):
        k = int(k)
        assert int(g["status"][k]) == int(r["status"][t]), f"LP {k}: status {g['status'][k]} vs oracle {r['status'][t]}"
        if int(r["status"][t]) == lpb.LP_OPTIMAL:
            go, ro = float(g["obj"][k]), float(r["obj"][t])
            assert abs(go - ro) <= OBJ_RTOL * max(1.0, abs(ro)), f"LP {k}: obj {go!r} vs oracle {ro!r}"


def test_headline_mixed_path_at_full_size():
    batch = W.WORKLOADS["dense50x50_phase1_100k"]()
    g = gpu_solve(batch, opts=mixed_opts())
    idx = sample(batch.num_lps, 600, seed=11)
    r = oracle_solve(batch, idx)
    check_status_obj(g, r, idx)
    st = g["status"]
    assert np.all(np.isin(st, [0, 1, 2]))
    assert np.all(st[batch.kind == W.KIND_INFEASIBLE] == lpb.LP_INFEASIBLE)
    assert np.all(st[batch.kind == W.KIND_UNBOUNDED] == lpb.LP_UNBOUNDED)
    A = batch.A.reshape(-1, 50, 50)
    b = batch.b.reshape(-1, 50)
    c = batch.c.reshape(-1, 50)
    x = g["x"].reshape(-1, 50)
    y = g["y"].reshape(-1, 50)
    opt = st == lpb.LP_OPTIMAL
    # optimal: primal feasible, c^T x = obj, slack duals >= 0, reduced costs
    # A^T y - c >= 0 (dual feasible), complementary: b^T y = c^T x
    viol = np.einsum("kij,kj->ki", A[opt], x[opt]) - b[opt]
    assert viol.max() <= 1e-8 * max(1.0, np.abs(b).max())
    assert x[opt].min() >= -1e-9
    np.testing.assert_allclose(np.einsum("kj,kj->k", c[opt], x[opt]), g["obj"][opt], rtol=1e-9, atol=1e-9)
    assert y[opt].min() >= -1e-9
    red = np.einsum("kij,ki->kj", A[opt], y[opt]) - c[opt]
    assert red.min() >= -1e-8
    np.testing.assert_allclose(np.einsum("ki,ki->k", b[opt], y[opt]), g["obj"][opt], rtol=1e-9, atol=1e-9)
    # infeasible: Farkas y >= 0, A^T y >= 0, b^T y < 0
    inf = st == lpb.LP_INFEASIBLE
    yi = y[inf]
    ys = np.maximum(1.0, np.abs(yi).max(axis=1))
    assert np.all(yi.min(axis=1) >= -1e-7 * ys)
    assert np.all(np.einsum("kij,ki->kj", A[inf], yi).min(axis=1) >= -1e-7 * ys)
    assert np.all(np.einsum("ki,ki->k", b[inf], yi) < 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_support_function_at_full_size(precision):
    batch = W.WORKLOADS["support40x10_100k"]()
    opts = mixed_opts() if precision == "fp32r" else None
    g = gpu_solve(batch, opts=opts)
    idx = sample(batch.num_lps, 1000, seed=12)
    r = oracle_solve(batch, idx)
    if precision == "fp64":
        n, bitwise = compare(batch, g, r, idx)
        assert bitwise == n
    else:
        check_status_obj(g, r, idx)
    # the polytope is bounded: every direction has a finite support value
    assert np.all(g["status"] == lpb.LP_OPTIMAL)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_uneven_batch_at_full_size(precision):
    batch = W.WORKLOADS["uneven10to500_20k"]()
    opts = mixed_opts() if precision == "fp32r" else None
    g = gpu_solve(batch, opts=opts)
    size = batch.m.astype(np.int64) * batch.n.astype(np.int64)
    largest = np.argsort(size)[-6:]          # tableaux in global memory on both paths
    idx = sample(batch.num_lps, 250, seed=13, extra=largest)
    r = oracle_solve(batch, idx)
    if precision == "fp64":
        n, bitwise = compare(batch, g, r, idx)
        assert bitwise == n
    else:
        check_status_obj(g, r, idx)
    # positive data: the slack basis is feasible and every LP is bounded
    assert np.all(g["status"] == lpb.LP_OPTIMAL)
