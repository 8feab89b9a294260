"""Pins of the CPU oracle against facts other than itself (CPU only).

The oracle is the plain FP64 tableau simplex of Section 3 of Gurung & Ray
(arXiv 1802.08557).  It is checked here against
  * hand-worked examples (tests/golden/worked_*.json),
  * brute-force vertex enumeration on tiny LPs (status and optimum),
  * closed forms: one constraint (m = 1), one variable (n = 1) and the
    hyper-rectangle LP of Eq. 7 (whose lower bounds > 0 exercise phase I),
  * LP duality certificates on every status (primal/dual feasibility and
    strong duality; Farkas multipliers; unbounded rays),
  * exact invariances (scaling b or c by a power of two),
and a mutation check shows that plausible mistakes in the oracle fail them.
"""
import ctypes
import glob
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from brute_force import brute_force

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "worked_*.json")))


@pytest.mark.parametrize("path", _golden_cases(), ids=lambda p: os.path.basename(p)[:-5])
def test_golden_worked_examples(path):
    g = json.load(open(path))
    r = oracle.solve(np.array(g["A"], float), np.array(g["b"], float), np.array(g["c"], float))
    assert r["status"] == g["status"]
    assert r["iters"] == g["iters"]
    assert r["phase1_iters"] == g["phase1_iters"]
    assert r["obj"] == pytest.approx(g["obj"], abs=1e-12)
    np.testing.assert_allclose(r["x"], g["x"], atol=1e-12)
    np.testing.assert_allclose(r["y"], g["y"], atol=1e-12)
    if "ray" in g:
        np.testing.assert_allclose(r["ray"], g["ray"], atol=1e-12)


def tiny_lps(seed, count):
    """Tiny LPs of three kinds: continuous mixed sign (all statuses), small
    integers (degenerate vertices and ties), and positive data (optimal)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        m = int(rng.integers(1, 7))
        n = int(rng.integers(1, 5))
        kind = t % 3
        if kind == 0:
            A = rng.uniform(-1, 1, (m, n))
            b = rng.uniform(-0.5, 2.0, m)
            c = rng.uniform(-1, 1, n)
        elif kind == 1:
            A = rng.integers(-2, 4, (m, n)).astype(float)
            b = rng.integers(-2, 5, m).astype(float)
            c = rng.integers(-2, 4, n).astype(float)
        else:
            A = rng.uniform(0.1, 1, (m, n))
            b = rng.uniform(0.5, 2, m)
            c = rng.uniform(0.1, 1, n)
        out.append((A, b, c))
    return out


def test_brute_force_agreement_tiny():
    counts = {0: 0, 1: 0, 2: 0}
    for A, b, c in tiny_lps(1234, 600):
        st, val = brute_force(A, b, c)
        r = oracle.solve(A, b, c)
        assert r["status"] == st, (A, b, c, r["status"], st)
        counts[st] += 1
        if st == 0:
            assert abs(r["obj"] - val) <= 1e-9 * max(1.0, abs(val)), (A, b, c, r["obj"], val)
    # every status occurs, so each branch is pinned
    assert min(counts.values()) >= 20, counts


def check_certificate(A, b, c, r, tol=1e-7):
    """LP duality certificates for the outcome ``r`` of max c^T x, Ax <= b, x >= 0."""
    x, y = r["x"], r["y"]
    scale = max(1.0, np.abs(A).max(), np.abs(b).max(), np.abs(c).max())
    st = r["status"]
    if st == oracle.OPTIMAL:
        assert np.all(x >= -tol * scale)
        assert np.all(A @ x <= b + tol * scale * (1 + np.abs(b)))
        assert np.all(y >= -tol * scale)
        assert np.all(A.T @ y >= c - tol * scale * (1 + np.abs(c)))
        p, d = float(c @ x), float(b @ y)
        assert abs(p - d) <= 1e-9 * max(1.0, abs(p)) * max(1.0, scale) * 10, (p, d)
        assert abs(p - r["obj"]) <= 1e-9 * max(1.0, abs(p)) * 10
    elif st == oracle.INFEASIBLE:
        assert np.all(y >= -tol)
        assert np.all(A.T @ y >= -tol * scale)
        assert float(b @ y) < -1e-9
    elif st == oracle.UNBOUNDED:
        d = r["ray"]
        assert np.all(d >= -tol)
        assert np.all(A @ d <= tol * scale)
        assert float(c @ d) > 1e-9
        # the current point is feasible too
        assert np.all(A @ x <= b + tol * scale * (1 + np.abs(b)))
    else:
        pytest.fail(f"unexpected status {st}")


def test_certificates_random_sizes():
    rng = np.random.default_rng(7)
    seen = set()
    for t in range(300):
        m = int(rng.integers(2, 30))
        n = int(rng.integers(2, 30))
        A = rng.uniform(-1, 1, (m, n))
        b = rng.uniform(-3, 10, m) if t % 2 else rng.uniform(1, 10, m)
        c = rng.uniform(-1, 1, n)
        r = oracle.solve(A, b, c)
        check_certificate(A, b, c, r)
        seen.add(r["status"])
    assert seen == {0, 1, 2}


def test_certificates_benchmark_shapes():
    from paper_1802_08557_gb300 import workloads as W
    for B in (W.positive_dense(50, 5, 5), W.mixed_sign_dense(300, 50, 50),
              W.support_function(50), W.uneven_dense(12, lo=10, hi=60),
              W.shared_matrix_family(4, m=60, n=30)):
        for k in range(B.num_lps):
            A, b, c = B.lp(k)
            r = oracle.solve(A, b, c)
            check_certificate(A, b, c, r)
            if B.kind[k] == W.KIND_INFEASIBLE:
                assert r["status"] == oracle.INFEASIBLE
            if B.kind[k] == W.KIND_UNBOUNDED:
                assert r["status"] == oracle.UNBOUNDED


def test_closed_form_single_constraint():
    """m = 1, from the one-row dual  min b*y  s.t.  a_j*y >= c_j, y >= 0:
    the dual feasible set is [ylo, yhi] with ylo = max(0, max_{a_j>0} c_j/a_j),
    yhi = min_{a_j<0} c_j/a_j (and c_j <= 0 wherever a_j = 0).  The primal is
    feasible iff b >= 0 or some a_j < 0.  Feasible primal + empty dual set ->
    unbounded; otherwise the optimum is b*ylo (b >= 0) or b*yhi (b < 0)."""
    rng = np.random.default_rng(11)
    seen = set()
    for t in range(600):
        n = int(rng.integers(1, 8))
        a = rng.uniform(-1, 1, n)
        a[rng.uniform(size=n) < 0.1] = 0.0
        c = rng.uniform(-1, 1, n)
        b = float(rng.uniform(-2, 3))
        r = oracle.solve(a[None, :], np.array([b]), c)
        seen.add(r["status"])
        if b < 0 and np.all(a >= 0):
            assert r["status"] == oracle.INFEASIBLE
            continue
        pos, neg = a > 0, a < 0
        ylo = max([0.0] + list(c[pos] / a[pos]))
        yhi = min([np.inf] + list(c[neg] / a[neg]))
        if np.any((a == 0) & (c > 0)) or ylo > yhi:
            assert r["status"] == oracle.UNBOUNDED
            continue
        assert r["status"] == oracle.OPTIMAL
        want = b * ylo if b >= 0 else b * yhi
        assert r["obj"] == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert seen == {0, 1, 2}


def test_closed_form_single_variable():
    """n = 1: the feasible set is an interval [lo, hi] of x >= 0."""
    rng = np.random.default_rng(12)
    for t in range(400):
        m = int(rng.integers(1, 7))
        a = rng.uniform(-1, 1, m)
        a[rng.uniform(size=m) < 0.15] = 0.0
        b = rng.uniform(-1, 2, m)
        c = float(rng.uniform(-1, 1))
        lo = max([0.0] + [b[i] / a[i] for i in range(m) if a[i] < 0])
        hi = min([np.inf] + [b[i] / a[i] for i in range(m) if a[i] > 0])
        zero_bad = any(a[i] == 0 and b[i] < 0 for i in range(m))
        r = oracle.solve(a[:, None], b, np.array([c]))
        if zero_bad or lo > hi + 1e-12:
            assert r["status"] == oracle.INFEASIBLE
        elif c > 0 and hi == np.inf:
            assert r["status"] == oracle.UNBOUNDED
        else:
            assert r["status"] == oracle.OPTIMAL
            want = c * hi if c > 0 else c * lo
            assert r["obj"] == pytest.approx(want, rel=1e-10, abs=1e-10)


def box_lp(lo, hi, ell):
    """Hyper-rectangle LP of Eq. 7 with free x = x+ - x-:
    x+ - x- <= hi and -(x+ - x-) <= -lo; objective (ell, -ell)."""
    d = len(lo)
    I = np.eye(d)
    A = np.block([[I, -I], [-I, I]])
    b = np.concatenate([hi, -lo])
    c = np.concatenate([ell, -ell])
    return A, b, c


def test_hyperbox_closed_form_eq7():
    """Eq. 7: max_{x in box} l.x = sum_i l_i h_i with h_i = lo_i if l_i < 0
    else hi_i.  Boxes with lo_i > 0 put negative entries in b: phase I."""
    rng = np.random.default_rng(13)
    saw_phase1 = 0
    for t in range(200):
        d = int(rng.integers(1, 9))
        lo = rng.uniform(-2, 2, d)
        hi = lo + rng.uniform(0.1, 3, d)
        ell = rng.standard_normal(d)
        A, b, c = box_lp(lo, hi, ell)
        r = oracle.solve(A, b, c)
        want = float(np.sum(np.where(ell < 0, lo, hi) * ell))
        assert r["status"] == oracle.OPTIMAL
        assert r["obj"] == pytest.approx(want, rel=1e-12, abs=1e-12)
        saw_phase1 += r["num_artificial"] > 0
    assert saw_phase1 > 50


def test_power_of_two_scaling_is_exact():
    """Multiplying c (or b) by 2 scales every reduced cost (or every RHS and
    ratio) exactly, so the pivot sequence, the iteration count and the scaled
    results must be bit-identical."""
    from paper_1802_08557_gb300 import workloads as W
    B = W.mixed_sign_dense(60, 20, 20)
    for k in range(B.num_lps):
        A, b, c = B.lp(k)
        r0 = oracle.solve(A, b, c)
        r1 = oracle.solve(A, b, 2.0 * c)
        assert r1["status"] == r0["status"] and r1["iters"] == r0["iters"]
        assert r1["obj"] == 2.0 * r0["obj"]
        np.testing.assert_array_equal(r1["x"], r0["x"])
        if r0["status"] != oracle.INFEASIBLE:
            np.testing.assert_array_equal(r1["y"], 2.0 * r0["y"])
        if r0["num_artificial"] == 0:  # b scaling also scales the tie windows' scale: keep to |ratios| <= 1 cases out
            r2 = oracle.solve(A, 0.5 * b, c)
            if r2["iters"] == r0["iters"]:
                assert r2["obj"] == 0.5 * r0["obj"]


def test_iteration_limit_and_count():
    g = json.load(open(os.path.join(GOLDEN, "worked_phase1_driveout.json")))
    A, b, c = (np.array(g[k], float) for k in ("A", "b", "c"))
    for lim in (1, 2, 3):
        r = oracle.solve(A, b, c, oracle.default_opts(max_iters=lim))
        assert r["status"] == oracle.ITER_LIMIT and r["iters"] == lim
    r = oracle.solve(A, b, c, oracle.default_opts(max_iters=4))
    assert r["status"] == oracle.OPTIMAL and r["iters"] == 4


# ---------------------------------------------------------------------------
# Mutation check: plausible mistakes planted in a copy of the oracle fail the pins
# ---------------------------------------------------------------------------

MUTATIONS = [
    ("update sign", "fma(-f, T(tb, l, j), T(tb, i, j))", "fma(f, T(tb, l, j), T(tb, i, j))"),
    ("entering argmax", "if (!found || d < dmin) { dmin = d; found = 1; }",
     "if (!found || d > dmin) { dmin = d; found = 1; }"),
    ("ratio argmax", "if (!found || r < rmin) { rmin = r; found = 1; }",
     "if (!found || r > rmin) { rmin = r; found = 1; }"),
    ("ratio eligibility dropped", "        if (!(a > o->eps_piv)) continue;\n        double r = T(tb, i, rhs) / a;\n        if (!found",
     "        if (a == 0.0) continue;\n        double r = T(tb, i, rhs) / a;\n        if (!found"),
    ("pivot row multiplied", "T(tb, l, j) = T(tb, l, j) / pe;", "T(tb, l, j) = T(tb, l, j) * pe;"),
    ("objective sign", "T(tb, m, j) = -c[j];", "T(tb, m, j) = c[j];"),
    ("row not negated", "for (int j = 0; j < tb->ncol; ++j) T(tb, i, j) = -T(tb, i, j);", ""),
    ("phase-I row added", "T(tb, w, j) = T(tb, w, j) - T(tb, i, j);", "T(tb, w, j) = T(tb, w, j) + T(tb, i, j);"),
    ("transposed A", "A[(size_t)i * (size_t)n + (size_t)j]", "A[(size_t)j * (size_t)m + (size_t)i]"),
    ("leaving tie takes last row", "        if (r <= thr) return i;\n", "        if (r <= thr && i + 1 == tb->m) return i;\n        if (r <= thr && 0) return i;\n"),
    ("drive-out skipped", "if (jsel < 0) continue; /* redundant row */", "continue;"),
    ("x from wrong column", "x[tb.basis[i]] = T(&tb, i, rhs);", "x[tb.basis[i]] = T(&tb, i, 0);"),
]


def _compile_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "simplex_oracle.c")).read()
    assert old in src, f"mutation anchor not found: {name}"
    mut = src.replace(old, new, 1)
    d = tmp_path / name.replace(" ", "_")
    d.mkdir()
    cfile = d / "simplex_oracle.c"
    cfile.write_text(mut)
    hdr = os.path.join(os.path.dirname(oracle.__file__), "simplex_oracle.h")
    (d / "simplex_oracle.h").write_text(open(hdr).read())
    so = d / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(cfile), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    L.oracle_solve.restype = ctypes.c_int
    L.oracle_solve.argtypes = oracle.lib().oracle_solve.argtypes
    return L


def _solve_with(L, A, b, c, max_iters=0):
    A = np.ascontiguousarray(A, float)
    b = np.ascontiguousarray(b, float)
    c = np.ascontiguousarray(c, float)
    m, n = A.shape
    x, y, ray = np.zeros(n), np.zeros(m), np.zeros(n)
    res = oracle.OracleResult()
    opts = oracle.default_opts(max_iters=max_iters or 200 * (m + n))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    L.oracle_solve(m, n, p(A), p(b), p(c), ctypes.byref(opts), ctypes.byref(res), p(x), p(y), p(ray))
    return dict(status=res.status, iters=res.iters, phase1_iters=res.phase1_iters, obj=res.obj,
                x=x, y=y, ray=ray, num_artificial=res.num_artificial)


def _pins_pass(L):
    """Quick version of the pins above against library L; False on first failure."""
    try:
        for path in _golden_cases():
            g = json.load(open(path))
            r = _solve_with(L, np.array(g["A"], float), np.array(g["b"], float), np.array(g["c"], float))
            if (r["status"] != g["status"] or r["iters"] != g["iters"]
                    or not np.allclose(r["x"], g["x"], atol=1e-12)
                    or not np.allclose(r["y"], g["y"], atol=1e-12)
                    or abs(r["obj"] - g["obj"]) > 1e-12):
                return False
        for A, b, c in tiny_lps(99, 150):
            st, val = brute_force(A, b, c)
            r = _solve_with(L, A, b, c)
            if r["status"] != st:
                return False
            if st == 0 and abs(r["obj"] - val) > 1e-9 * max(1.0, abs(val)):
                return False
        rng = np.random.default_rng(5)
        for t in range(40):
            d = int(rng.integers(1, 6))
            lo = rng.uniform(-2, 2, d)
            hi = lo + rng.uniform(0.1, 3, d)
            ell = rng.standard_normal(d)
            r = _solve_with(L, *box_lp(lo, hi, ell))
            if r["status"] != 0 or abs(r["obj"] - float(np.sum(np.where(ell < 0, lo, hi) * ell))) > 1e-9:
                return False
    except Exception:
        return False
    return True


def test_unmutated_oracle_passes_quick_pins(tmp_path):
    L = _compile_mutant(tmp_path, "identity", "fma(-f,", "fma(-f,")
    assert _pins_pass(L)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    L = _compile_mutant(tmp_path, name, old, new)
    assert not _pins_pass(L), f"mutation '{name}' survived the pins"
