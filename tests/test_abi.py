"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; argument errors are reported as codes before any device work
(CPU only: no GPU call is made here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1802_08557_gb300 import build as B
from paper_1802_08557_gb300 import lpbatch as lpb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lpb.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"lp_batch_create", "lp_batch_solve", "lp_batch_results", "lp_batch_destroy"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(lpb.EXPORTED) == names


def test_sm103a_only_build():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_strerror_and_defaults(lib):
    for code in range(6):
        assert lpb.strerror(code)
    o = lpb.lpb_default_opts()
    assert o.eps_opt == 1e-9 and o.eps_piv == 1e-9 and o.eps_feas == 1e-9 and o.tau == 1e-12
    assert o.max_iters == 0 and o.precision == lpb.LP_PREC_FP64


def _create_raw(lib, num, m, n, A, b, c, ptr_kind=lpb.LPB_HOST, a_len=None):
    h = ctypes.c_void_p()
    mm = np.ascontiguousarray(m, np.int32)
    nn = np.ascontiguousarray(n, np.int32)
    return lib.lp_batch_create(ctypes.byref(h), num, mm.ctypes.data, nn.ctypes.data,
                               None, A.ctypes.data if A is not None else None,
                               a_len if a_len is not None else (A.size if A is not None else 0),
                               None, b.ctypes.data if b is not None else None, b.size if b is not None else 0,
                               None, c.ctypes.data if c is not None else None, c.size if c is not None else 0,
                               ptr_kind, None, None), h


def test_argument_errors_before_device_work(lib):
    A, b, c = np.ones(4), np.ones(2), np.ones(2)
    assert lib.lp_batch_create(None, 1, None, None, None, None, 0, None, None, 0, None, None, 0, 0, None, None) == lpb.LPB_EINVAL
    code, h = _create_raw(lib, 0, [2], [2], A, b, c)
    assert code == lpb.LPB_EINVAL and not h.value
    code, h = _create_raw(lib, 1, [0], [2], A, b, c)
    assert code == lpb.LPB_EINVAL
    code, h = _create_raw(lib, 1, [2], [2], None, b, c)
    assert code == lpb.LPB_EINVAL
    code, h = _create_raw(lib, 1, [2], [2], A, b, c, ptr_kind=7)
    assert code == lpb.LPB_EINVAL
    code, h = _create_raw(lib, 1, [2], [2], A, b, c, a_len=3)  # A too short for 2x2
    assert code == lpb.LPB_EINVAL
    assert b"A offset" in lib.lpb_last_error()
    code, h = _create_raw(lib, 1, [lpb.LPB_MAX_DIM + 1], [2], A, b, c)
    assert code == lpb.LPB_ETOOBIG
    assert lib.lp_batch_solve(None, None) == lpb.LPB_EINVAL
    assert lib.lp_batch_results(None, None, None, None, None, None, 0) == lpb.LPB_EINVAL
    assert lib.lp_batch_destroy(None) == lpb.LPB_OK


def test_solve_host_argument_errors_before_device_work(lib):
    A, b, c = np.ones(4), np.ones(2), np.ones(2)
    m, n = np.array([2], np.int32), np.array([2], np.int32)
    st, it, ob, x = np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1), np.zeros(2)
    P = lambda a: a.ctypes.data if a is not None else None

    def call(num=1, mm=m, AA=A, a_len=4, chunks=0, xx=x):
        return lib.lp_solve_host(num, P(mm), P(n), None, P(AA), a_len, None, P(b), 2, None, P(c), 2, None, chunks,
                                 P(st), P(it), P(ob), P(xx), None)
    assert call(num=0) == lpb.LPB_EINVAL
    assert call(AA=None) == lpb.LPB_EINVAL
    assert call(xx=None) == lpb.LPB_EINVAL
    assert call(chunks=-1) == lpb.LPB_EINVAL
    assert call(chunks=65) == lpb.LPB_EINVAL
    assert call(mm=np.array([0], np.int32)) == lpb.LPB_EINVAL
    assert call(a_len=3) == lpb.LPB_EINVAL
    assert b"offset out of range" in lib.lpb_last_error()


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(lpb, "_lib", None)
    with pytest.raises(ImportError):
        lpb.load(str(tmp_path / "missing.so"))


def test_hyperbox_argument_errors_before_device_work(lib):
    L, lo, hi, obj = np.ones(8), np.zeros(4), np.ones(4), np.zeros(2)
    args = lambda num, dim, Lp=L.ctypes.data, kind=lpb.LPB_HOST: (num, dim, lo.ctypes.data, hi.ctypes.data, 0, Lp,
                                                                    obj.ctypes.data, None, kind, None)
    assert lib.lp_hyperbox_solve(*args(2, 0)) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(*args(-1, 4)) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(*args(2, (1 << 20) + 1)) == lpb.LPB_ETOOBIG
    assert lib.lp_hyperbox_solve(*args(2, 4, Lp=None)) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(*args(2, 4, kind=9)) == lpb.LPB_EINVAL
    assert lib.lp_hyperbox_solve(*args(0, 4)) == lpb.LPB_OK  # empty batch: nothing to do


def test_mlp_argument_errors_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.lp_mlp_create(None, 4, 4, 4, 4, 8, 0) == lpb.LPB_EINVAL
    assert lib.lp_mlp_create(ctypes.byref(h), 0, 4, 4, 4, 8, 0) == lpb.LPB_EINVAL
    assert lib.lp_mlp_create(ctypes.byref(h), 4, 4, 4, 4, 0, 0) == lpb.LPB_EINVAL
    assert lib.lp_mlp_create(ctypes.byref(h), 1 << 14, 4, 4, 4, 8, 0) == lpb.LPB_ETOOBIG
    assert not h.value
    assert lib.lp_mlp_destroy(None) == lpb.LPB_OK
