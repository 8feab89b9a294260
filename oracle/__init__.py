"""CPU FP64 reference (oracle) of the dense two-phase simplex of Gurung & Ray,
"Simultaneous Solving of Batched Linear Programs on a GPU" (arXiv 1802.08557),
Section 3 (Eq. 1-4, Steps 1-3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA solver in
``paper_1802_08557_gb300`` never imports it, and the two share no code.

The arithmetic lives in ``simplex_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so that only the explicit ``fma`` of the pivot update is
fused).  This module builds it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "libsimplex_oracle.so")

OPTIMAL, INFEASIBLE, UNBOUNDED, ITER_LIMIT, NUMERICAL = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "optimal", 1: "infeasible", 2: "unbounded", 3: "iter_limit", 4: "numerical"}


class OracleOpts(ctypes.Structure):
    _fields_ = [
        ("eps_opt", ctypes.c_double),
        ("eps_piv", ctypes.c_double),
        ("eps_feas", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("max_iters", ctypes.c_int32),
    ]


class OracleResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("phase1_iters", ctypes.c_int32),
        ("num_artificial", ctypes.c_int32),
        ("entering", ctypes.c_int32),
        ("obj", ctypes.c_double),
        ("phase1_obj", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` with gcc (no GPU needed)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_solve.restype = ctypes.c_int
            L.oracle_solve.argtypes = [
                ctypes.c_int32, ctypes.c_int32,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.POINTER(OracleOpts), ctypes.POINTER(OracleResult),
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ]
            L.oracle_default_opts.argtypes = [ctypes.POINTER(OracleOpts)]
            L.oracle_default_opts.restype = None
            _lib = L
    return _lib


def default_opts(**kw) -> OracleOpts:
    o = OracleOpts()
    lib().oracle_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def solve(A, b, c, opts: OracleOpts | None = None) -> dict:
    """Solve max c^T x s.t. A x <= b, x >= 0 (Eq. 1-3) with the two-phase
    tableau simplex.  Returns status, iters, phase1_iters, obj (tableau
    corner), x, y (slack reduced costs: duals, or Farkas multipliers when
    infeasible), ray (unbounded direction) and num_artificial."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m, n = A.shape
    assert b.shape == (m,) and c.shape == (n,)
    if opts is None:
        opts = default_opts()
    x = np.zeros(n)
    y = np.zeros(m)
    ray = np.zeros(n)
    r = OracleResult()
    rc = lib().oracle_solve(m, n, _ptr(A), _ptr(b), _ptr(c), ctypes.byref(opts),
                            ctypes.byref(r), _ptr(x), _ptr(y), _ptr(ray))
    if rc != 0:
        raise RuntimeError(f"oracle_solve failed with code {rc}")
    return dict(status=r.status, iters=r.iters, phase1_iters=r.phase1_iters,
                num_artificial=r.num_artificial, entering=r.entering,
                obj=r.obj, phase1_obj=r.phase1_obj, x=x, y=y, ray=ray)


def solve_batch(lps, opts: OracleOpts | None = None, threads: int = 1) -> dict:
    """Solve a list of (A, b, c) one by one.  With ``threads > 1`` the LPs are
    spread over a thread pool (ctypes releases the GIL during each call)."""
    if opts is None:
        opts = default_opts()
    N = len(lps)
    status = np.zeros(N, np.int32)
    iters = np.zeros(N, np.int32)
    obj = np.zeros(N)
    xs = [None] * N
    ys = [None] * N

    def one(k):
        A, b, c = lps[k]
        r = solve(A, b, c, opts)
        status[k] = r["status"]
        iters[k] = r["iters"]
        obj[k] = r["obj"]
        xs[k] = r["x"]
        ys[k] = r["y"]

    lib()
    if threads <= 1:
        for k in range(N):
            one(k)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, range(N), chunksize=max(1, N // (threads * 8))))
    return dict(status=status, iters=iters, obj=obj, x=xs, y=ys)
