"""The oracle against an independent LP solver (HiGHS through scipy's
linprog) on LPs of the benchmark shapes: the same status, and the same
optimum within 1e-7 relative where one exists.  A wrong pivot rule, sign or
phase-I step in the oracle changes one of these on some LP.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1802_08557_gb300 import workloads as W

linprog = pytest.importorskip("scipy.optimize").linprog

# linprog status: 0 optimal, 2 infeasible, 3 unbounded
HIGHS_TO_ORACLE = {0: oracle.OPTIMAL, 2: oracle.INFEASIBLE, 3: oracle.UNBOUNDED}


def _check(batch, count):
    seen = set()
    for k in range(min(count, batch.num_lps)):
        A, b, c = batch.lp(k)
        r = oracle.solve(A, b, c)
        h = linprog(-c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
        assert h.status in HIGHS_TO_ORACLE, (k, h.message)
        assert r["status"] == HIGHS_TO_ORACLE[h.status], (batch.name, k, r["status"], h.status)
        seen.add(r["status"])
        if h.status == 0:
            ref = -h.fun
            assert abs(r["obj"] - ref) <= 1e-7 * max(1.0, abs(ref)), (batch.name, k, r["obj"], ref)
    return seen


def test_mixed_sign_dense_50x50():
    # phase-I, infeasible and unbounded LPs all occur in the first 120
    assert _check(W.mixed_sign_dense(120), 120) == {oracle.OPTIMAL, oracle.INFEASIBLE, oracle.UNBOUNDED}


def test_other_benchmark_shapes():
    _check(W.positive_dense(40, 5, 5), 40)
    _check(W.support_function(40), 40)
    _check(W.uneven_dense(6, lo=10, hi=80), 6)
    _check(W.shared_matrix_family(6, m=60, n=30), 6)


def test_degenerate_and_phase1_heavy():
    """Many ties and negative right-hand sides: b from a few integers, A
    integer-valued."""
    rng = np.random.default_rng(3)
    lps = []
    for _ in range(60):
        m, n = int(rng.integers(3, 12)), int(rng.integers(3, 12))
        A = rng.integers(-3, 4, size=(m, n)).astype(float)
        b = rng.integers(-2, 5, size=m).astype(float)
        c = rng.integers(-2, 4, size=n).astype(float)
        lps.append((A, b, c))
    _check(W.pack("integer_degenerate", lps), 60)
