"""Pins of the synthetic input recipes: each generator draws what its recipe
states (value ranges, the phase-I and constructed fractions of the dense
random LPs, log-uniform sizes of the uneven batch, unit normals and shared
data of the support-function polytope, the shared matrix family), the batch
layout is consistent, and any LP regenerates alone from its index.  CPU only.

The constructed infeasible and unbounded LPs are checked against the
mathematical certificate their construction plants (a pair of opposite rows
with incompatible right-hand sides; a column with no positive entry and a
positive cost at a feasible origin), not against any solver."""
import math

import numpy as np
import pytest

from paper_1802_08557_gb300 import workloads as W


def _check_layout(B: W.LPBatch):
    N = B.num_lps
    assert B.m.dtype == np.int32 and B.n.dtype == np.int32
    for off in (B.a_off, B.b_off, B.c_off):
        assert off.dtype == np.int64 and off.shape == (N,)
    assert B.A.dtype == np.float64 and B.b.dtype == np.float64 and B.c.dtype == np.float64
    mn = B.m.astype(np.int64) * B.n.astype(np.int64)
    assert np.all(B.a_off >= 0) and np.all(B.a_off + mn <= B.A.size)
    assert np.all(B.b_off >= 0) and np.all(B.b_off + B.m <= B.b.size)
    assert np.all(B.c_off >= 0) and np.all(B.c_off + B.n <= B.c.size)
    assert B.kind.shape == (N,)
    assert np.all(np.isfinite(B.A)) and np.all(np.isfinite(B.b)) and np.all(np.isfinite(B.c))


def test_positive_dense_ranges_and_layout():
    """Section 5's positive random LPs: A~U[1,10], b~U[10,100], c~U[1,10]."""
    B = W.positive_dense(300, 5, 5)
    _check_layout(B)
    assert np.all(B.m == 5) and np.all(B.n == 5)
    assert np.array_equal(B.a_off, np.arange(300) * 25)
    assert B.A.min() >= 1.0 and B.A.max() < 10.0
    assert B.b.min() >= 10.0 and B.b.max() < 100.0
    assert B.c.min() >= 1.0 and B.c.max() < 10.0
    # uniform, not clustered at one end: the mean of U[lo,hi] within 3%
    assert abs(B.A.mean() - 5.5) < 0.15
    assert abs(B.b.mean() - 55.0) < 1.5
    assert np.all(B.kind == W.KIND_FEASIBLE_START)


def test_lp_regenerates_alone_from_its_index():
    """Each LP has its own counter-based generator: LP i of a batch started at
    s equals LP s+i of a batch started at 0, for every generator."""
    pairs = [
        (W.positive_dense(30, 5, 5), W.positive_dense(4, 5, 5, start=17), 17),
        (W.mixed_sign_dense(30, 20, 20), W.mixed_sign_dense(4, 20, 20, start=17), 17),
        (W.uneven_dense(30, lo=10, hi=40), W.uneven_dense(4, lo=10, hi=40, start=17), 17),
        (W.support_function(30), W.support_function(4, start=17), 17),
        (W.shared_matrix_family(30, m=20, n=10), W.shared_matrix_family(4, m=20, n=10, start=17), 17),
    ]
    for full, part, s in pairs:
        for i in range(part.num_lps):
            for u, v in zip(full.lp(s + i), part.lp(i)):
                assert np.array_equal(u, v)
            assert full.kind[s + i] == part.kind[i]
    # and LPs of different indices or workloads differ
    B = W.positive_dense(2, 5, 5)
    assert not np.array_equal(B.lp(0)[0], B.lp(1)[0])
    assert not np.array_equal(W.positive_dense(1, 5, 5, wid=7).A, B.lp(0)[0].ravel())


def test_hyperbox_directions_regenerate_by_block():
    L, lo, hi = W.hyperbox_directions(3 * 4096 + 5)
    L2, lo2, hi2 = W.hyperbox_directions(4096 + 5, start=2 * 4096)
    assert np.array_equal(L[2 * 4096:], L2)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)


def test_mixed_sign_dense_fractions_and_constructions():
    """The benchmark's 50x50 LPs: A, c ~ U[-1,1]; 20% draw b ~ U[-5,10] (then
    some b_i < 0 with probability 1 - (2/3)^50: phase I), the rest b ~ U[1,10],
    of which 2.5% (of all LPs) are made infeasible and 2.5% unbounded."""
    N = 4000
    B = W.mixed_sign_dense(N)
    _check_layout(B)
    assert np.all(B.m == 50) and np.all(B.n == 50)
    assert B.A.min() >= -1.0 and B.A.max() < 1.0
    assert B.c.min() >= -1.0 and B.c.max() <= 1.0
    frac = {k: float(np.mean(B.kind == k)) for k in range(4)}
    # binomial standard deviations at N = 4000: 0.0063 (p=.2), 0.0025 (p=.025)
    assert abs(frac[W.KIND_PHASE1] - 0.20) < 0.03
    assert abs(frac[W.KIND_INFEASIBLE] - 0.025) < 0.0125
    assert abs(frac[W.KIND_UNBOUNDED] - 0.025) < 0.0125
    n_inf = n_unb = 0
    for k in range(N):
        A, b, c = B.lp(k)
        kind = B.kind[k]
        if kind == W.KIND_PHASE1:
            assert b.min() < 0 and b.min() >= -5.0 and b.max() < 10.0
            continue
        if kind == W.KIND_INFEASIBLE:
            # one pair of rows a_k = -a_j with b_j + b_k in [-1, -0.5]:
            # a_j x <= b_j and a_j x >= b_j + delta cannot both hold
            neg = np.flatnonzero(b < 0)
            assert neg.size == 1
            kk = int(neg[0])
            j = [r for r in range(50) if r != kk and np.array_equal(A[r], -A[kk])]
            assert len(j) == 1
            j = j[0]
            assert 1.0 <= b[j] < 4.0 and -1.0 <= b[j] + b[kk] <= -0.5
            n_inf += 1
            continue
        # feasible origin: b ~ U[1,10]
        assert b.min() >= 1.0 and b.max() < 10.0
        if kind == W.KIND_UNBOUNDED:
            # a ray: column j has no positive entry and c_j > 0, the origin is feasible
            cols = [j for j in range(50) if np.all(A[:, j] <= 0) and c[j] >= 0.5]
            assert len(cols) >= 1
            n_unb += 1
    assert n_inf > 0 and n_unb > 0


def test_mixed_sign_dense_phase1_draws_negative_rhs_almost_always():
    """With b ~ U[-5,10], a 50-row LP has no negative b_i with probability
    (2/3)^50 < 2e-9: every LP drawn for phase I is tagged KIND_PHASE1, and
    no LP with a feasible origin has a negative b_i."""
    B = W.mixed_sign_dense(2000)
    neg_any = np.array([(B.lp(k)[1] < 0).any() for k in range(B.num_lps)])
    # the constructed infeasible LPs carry their one negative b_k as well
    assert np.array_equal(neg_any, (B.kind == W.KIND_PHASE1) | (B.kind == W.KIND_INFEASIBLE))
    assert (2.0 / 3.0) ** 50 < 2e-9


def test_uneven_sizes_are_log_uniform():
    """m, n = floor(exp(U[ln 10, ln 500])): every size in [10, 499]; half the
    draws below the geometric mean sqrt(10*500) ~ 70.7 (a uniform draw on
    [10, 500] would put only 12% there); m and n drawn independently."""
    B = W.uneven_dense(400)
    _check_layout(B)
    for s in (B.m, B.n):
        assert s.min() >= 10 and s.max() <= 499
        assert abs(float(np.mean(s < 71)) - (math.log(71) - math.log(10)) / math.log(50)) < 0.1
        # each third of [ln 10, ln 500) holds about a third of the draws
        t = np.floor(3 * (np.log(s) - math.log(10)) / math.log(50)).astype(int)
        for i in range(3):
            assert abs(float(np.mean(t == i)) - 1 / 3) < 0.1
    assert abs(float(np.corrcoef(np.log(B.m), np.log(B.n))[0, 1])) < 0.2
    assert B.A.min() >= 0.0 and B.A.max() < 1.0
    assert B.b.min() >= 1.0 and B.b.max() < 100.0
    assert B.c.min() >= 0.0 and B.c.max() < 1.0
    mn = B.m.astype(np.int64) * B.n.astype(np.int64)
    assert np.array_equal(B.a_off, np.concatenate([[0], np.cumsum(mn)[:-1]]))
    assert B.A.size == int(mn.sum())


def test_uneven_max_elems_caps_the_tableau():
    B = W.uneven_dense(200, max_elems=5000)
    assert np.all(B.m.astype(np.int64) * B.n <= 5000)
    assert B.m.min() >= 10 and B.n.min() >= 10


def test_support_function_polytope():
    """One polytope {z : a_i.z <= b_i} in R^10 with 40 unit normals and
    b ~ U[1,2] (origin interior); z = x+ - x- gives A = [a, -a] and c = [l, -l]
    with l a unit direction.  A and b are stored once and shared."""
    B = W.support_function(500)
    _check_layout(B)
    assert np.all(B.m == 40) and np.all(B.n == 20)
    assert np.all(B.a_off == 0) and np.all(B.b_off == 0)
    assert B.A.size == 40 * 20 and B.b.size == 40
    A, b, _ = B.lp(0)
    a = A[:, :10]
    assert np.array_equal(A[:, 10:], -a)
    assert np.allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-14)
    assert b.min() >= 1.0 and b.max() < 2.0
    # bounded: 0 = sum_i lam_i a_i with every lam_i > 0 (and the a_i spanning
    # R^10) means no direction l has a_i.l <= 0 for all i.  Checked by
    # max t  s.t.  a^T lam = 0, sum lam = 1, lam_i >= t.
    assert np.linalg.matrix_rank(a) == 10
    linprog = pytest.importorskip("scipy.optimize").linprog
    A_eq = np.vstack([np.hstack([a.T, np.zeros((10, 1))]), np.hstack([np.ones((1, 40)), [[0.0]]])])
    b_eq = np.concatenate([np.zeros(10), [1.0]])
    A_ub = np.hstack([-np.eye(40), np.ones((40, 1))])
    res = linprog(np.concatenate([np.zeros(40), [-1.0]]), A_ub=A_ub, b_ub=np.zeros(40), A_eq=A_eq,
                  b_eq=b_eq, bounds=[(0, None)] * 40 + [(None, None)])
    assert res.status == 0 and -res.fun > 1e-4
    C = B.c.reshape(500, 20)
    assert np.array_equal(C[:, 10:], -C[:, :10])
    assert np.allclose(np.linalg.norm(C[:, :10], axis=1), 1.0, atol=1e-14)
    # directions uniform on the sphere: mean near 0, second moment near I/10
    L = C[:, :10]
    assert np.abs(L.mean(axis=0)).max() < 0.1
    assert np.abs(L.T @ L / 500 - np.eye(10) / 10).max() < 0.05


def test_shared_matrix_family():
    """Shared A (200x100, U[0,1]) and b0 ~ U[1,100]; per LP b = b0 (1 + 0.1 N(0,1))
    and c ~ U[0,1].  Over many LPs the mean of b_i estimates b0_i and the
    relative spread is 0.1."""
    N = 3000
    B = W.shared_matrix_family(N)
    _check_layout(B)
    assert np.all(B.a_off == 0) and B.A.size == 200 * 100
    assert B.A.min() >= 0.0 and B.A.max() < 1.0
    Bm = B.b.reshape(N, 200)
    b0 = Bm.mean(axis=0)
    assert b0.min() > 0.9 and b0.max() < 101.0
    rel = Bm / b0 - 1.0
    assert abs(float(rel.std()) - 0.1) < 0.005
    assert abs(float(rel.mean())) < 0.002
    # normal, not uniform: kurtosis 3 (a uniform draw has 1.8)
    z = rel.ravel() / rel.std()
    assert abs(float(np.mean(z ** 4)) - 3.0) < 0.15
    C = B.c.reshape(N, 100)
    assert C.min() >= 0.0 and C.max() < 1.0
    assert np.array_equal(B.kind, np.where((Bm < 0).any(axis=1), W.KIND_PHASE1, W.KIND_FEASIBLE_START))


def test_shared_matrix_blocks_same_family_other_draws():
    """The training form shares A and b0 with the per-LP form but draws its
    own b and c (keyed apart), block by block."""
    P = W.shared_matrix_family(50, m=30, n=20)
    Q = W.shared_matrix_family_blocks(50, m=30, n=20)
    _check_layout(Q)
    assert np.array_equal(P.A, Q.A)
    assert not np.any(np.all(P.b.reshape(50, 30) == Q.b.reshape(50, 30), axis=1))
    R = W.shared_matrix_family_blocks(4096 + 7, m=30, n=20)
    S = W.shared_matrix_family_blocks(7, m=30, n=20, start=4096)
    assert np.array_equal(R.b[4096 * 30:], S.b) and np.array_equal(R.c[4096 * 20:], S.c)


def test_hyperbox_box_and_directions():
    """Box lo ~ U[-2,0], hi = lo + U[0.5,3]; directions unit vectors of R^28."""
    L, lo, hi = W.hyperbox_directions(5000)
    assert L.shape == (5000, 28) and lo.shape == (28,) and hi.shape == (28,)
    assert lo.min() >= -2.0 and lo.max() < 0.0
    w = hi - lo
    assert w.min() >= 0.5 and w.max() < 3.0
    assert np.allclose(np.linalg.norm(L, axis=1), 1.0, atol=1e-14)
    assert np.abs(L.mean(axis=0)).max() < 0.05
    assert np.abs(L.T @ L / 5000 - np.eye(28) / 28).max() < 0.01


def test_named_workloads_sizes():
    """The named benchmark workloads at a few LPs each: the sizes their names state."""
    want = {"dense5x5_1k": (5, 5), "dense50x50_phase1_100k": (50, 50), "support40x10_100k": (40, 20),
            "shared200x100_100k": (200, 100)}
    for name, (m, n) in want.items():
        B = W.WORKLOADS[name](num=3)
        assert B.num_lps == 3 and np.all(B.m == m) and np.all(B.n == n)
    U = W.WORKLOADS["uneven10to500_20k"](num=3)
    assert U.num_lps == 3 and U.m.min() >= 10 and U.n.max() <= 499
