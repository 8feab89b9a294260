"""Pins of the hyperbox oracle (Section 4.4, Eq. 7) against things other than
itself: the simplex oracle on the same LP written as Ax <= b, brute-force
enumeration of the box's vertices, exact integer cases, and the degenerate
cases the formula has.  A mutation check plants plausible mistakes into a copy
of the oracle and shows that each one fails these pins."""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import hyperbox

_SRC = os.path.join(os.path.dirname(oracle.__file__), "hyperbox.py")


def _box_lp(lo, hi, ell):
    """max ell.x over lo <= x <= hi as a standard-form LP (x = x+ - x-):
    x+ - x- <= hi, -(x+ - x-) <= -lo, objective (ell, -ell)."""
    d = len(lo)
    I = np.eye(d)
    A = np.block([[I, -I], [-I, I]])
    return A, np.concatenate([hi, -lo]), np.concatenate([ell, -ell])


def _vertex_max(lo, hi, ell):
    """max over the 2^d vertices of the box of ell.v, and the set of maximisers."""
    best, arg = None, []
    for bits in itertools.product((0, 1), repeat=len(lo)):
        v = np.where(np.array(bits) == 1, hi, lo)
        val = float(np.dot(ell, v))
        if best is None or val > best + 1e-12 * max(1.0, abs(best)):
            best, arg = val, [v]
        elif abs(val - best) <= 1e-12 * max(1.0, abs(best)):
            arg.append(v)
    return best, arg


# ---- the pins, as functions of a candidate implementation -----------------

def _pin_vs_simplex(fn):
    rng = np.random.default_rng(21)
    for _ in range(120):
        d = int(rng.integers(1, 8))
        lo = rng.uniform(-3, 3, d)
        hi = lo + rng.uniform(0.0, 4, d)
        ell = rng.standard_normal(d)
        obj, x = fn(ell[None, :], lo, hi)
        r = oracle.solve(*_box_lp(lo, hi, ell))
        assert r["status"] == oracle.OPTIMAL
        assert obj[0] == pytest.approx(r["obj"], rel=1e-10, abs=1e-10)
        assert np.all(x[0] >= lo) and np.all(x[0] <= hi)
        assert float(np.dot(ell, x[0])) == pytest.approx(obj[0], rel=1e-12, abs=1e-12)


def _pin_vs_vertices(fn):
    rng = np.random.default_rng(22)
    for _ in range(200):
        d = int(rng.integers(1, 7))
        lo = rng.uniform(-2, 2, d)
        hi = lo + rng.uniform(0.0, 2, d)
        ell = rng.uniform(-1, 1, d)
        ell[rng.random(d) < 0.15] = 0.0
        obj, x = fn(ell[None, :], lo, hi)
        best, arg = _vertex_max(lo, hi, ell)
        assert obj[0] == pytest.approx(best, rel=1e-12, abs=1e-12)
        assert any(np.array_equal(x[0], v) for v in arg)


def _pin_integer_exact(fn):
    rng = np.random.default_rng(23)
    L = rng.integers(-50, 51, (500, 9)).astype(np.float64)
    lo = rng.integers(-20, 1, 9).astype(np.float64)
    hi = lo + rng.integers(0, 30, 9)
    obj, x = fn(L, lo, hi)
    want = np.array([max(int(np.dot(l.astype(np.int64), v.astype(np.int64)))
                         for v in (np.where(np.array(bits) == 1, hi, lo)
                                   for bits in itertools.product((0, 1), repeat=9))) for l in L[:40]])
    np.testing.assert_array_equal(obj[:40], want)
    exact = (L.astype(np.int64) * np.where(L < 0, lo, hi).astype(np.int64)).sum(axis=1)
    np.testing.assert_array_equal(obj, exact.astype(np.float64))


def _pin_special_cases(fn):
    lo = np.array([-1.0, 2.0, -3.5])
    hi = np.array([4.0, 2.0, 0.5])
    # zero direction: value 0, maximiser = hi (the "otherwise" branch of Eq. 7)
    obj, x = fn(np.zeros((1, 3)), lo, hi)
    assert obj[0] == 0.0 and np.array_equal(x[0], hi)
    # a coordinate direction picks one bound
    for i in range(3):
        for s in (1.0, -1.0):
            e = np.zeros((1, 3))
            e[0, i] = s
            obj, x = fn(e, lo, hi)
            assert obj[0] == (hi[i] if s > 0 else -lo[i])
    # per-LP boxes: each row uses its own box
    L = np.array([[1.0, -1.0, 2.0], [-2.0, 0.5, -1.0]])
    los = np.array([[0.0, 1.0, -1.0], [-3.0, -3.0, -3.0]])
    his = np.array([[1.0, 2.0, 1.0], [3.0, 3.0, 3.0]])
    obj, x = fn(L, los, his)
    assert obj[0] == 1.0 - 1.0 + 2.0 and obj[1] == 6.0 + 1.5 + 3.0
    # a point box: every direction gives ell.lo
    obj, _ = fn(np.array([[3.0, -2.0, 1.0]]), hi, hi)
    assert obj[0] == 3.0 * 4.0 - 2.0 * 2.0 + 0.5


PINS = (_pin_vs_simplex, _pin_vs_vertices, _pin_integer_exact, _pin_special_cases)


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_meets_pin(pin):
    pin(hyperbox.hyperbox_solve)


# ---- mutation check ------------------------------------------------------

MUTATIONS = {
    "sign test reversed": ("np.where(L < 0.0, lo, hi)", "np.where(L > 0.0, lo, hi)"),
    "bounds swapped": ("np.where(L < 0.0, lo, hi)", "np.where(L < 0.0, hi, lo)"),
    "zero goes to lo": ("np.where(L < 0.0, lo, hi)", "np.where(L <= 0.0, lo, hi)"),
    "last term dropped": ("for i in range(L.shape[1]):", "for i in range(L.shape[1] - 1):"),
    "product sign": ("obj = obj + L[:, i] * h[:, i]", "obj = obj - L[:, i] * h[:, i]"),
    "lower box only": ("hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), L.shape)",
                       "hi = np.broadcast_to(np.asarray(lo, dtype=np.float64), L.shape)"),
    "first coordinate reused": ("obj = obj + L[:, i] * h[:, i]", "obj = obj + L[:, 0] * h[:, i]"),
}


def _mutant(old, new):
    src = open(_SRC).read()
    assert old in src, old
    ns = {}
    exec(compile(src.replace(old, new), "hyperbox_mutant", "exec"), ns)
    return ns["hyperbox_solve"]


def _passes_all(fn):
    for pin in PINS:
        try:
            pin(fn)
        except AssertionError:
            return False
    return True


def test_unmutated_copy_passes():
    assert _passes_all(_mutant("import numpy as np", "import numpy as np"))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert not _passes_all(_mutant(*MUTATIONS[name])), f"mutation '{name}' survived the pins"
