"""Thin ctypes binding of the C ABI in ``include/lpbatch.h``.

Names follow the C functions.  The binding only marshals arguments: every
step of the solve runs in the CUDA library.  Device buffers and streams come
from PyTorch (``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``);
host buffers are numpy arrays.  If the compiled library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LP_OPTIMAL, LP_INFEASIBLE, LP_UNBOUNDED, LP_ITER_LIMIT, LP_NUMERICAL = 0, 1, 2, 3, 4
LPB_OK, LPB_EINVAL, LPB_ENOMEM, LPB_ECUDA, LPB_ETOOBIG, LPB_ENOTSOLVED = 0, 1, 2, 3, 4, 5
LPB_HOST, LPB_DEVICE = 0, 1
LP_PREC_FP64, LP_PREC_FP32_REFINE = 0, 1
LPB_SCHED_AUTO, LPB_SCHED_STREAMED, LPB_SCHED_CLUSTER, LPB_SCHED_SINGLE = 0, 1, 2, 3
LPB_MAX_DIM = 16384
LPB_EPI_STORE, LPB_EPI_BIAS_RELU, LPB_EPI_BIAS, LPB_EPI_MASK_GRAD = 0, 1, 2, 3
LPB_GEMM_AUTO, LPB_GEMM_MMA64, LPB_GEMM_MMA128, LPB_GEMM_TC = 0, 1, 2, 3

# Every symbol include/lpbatch.h declares.
EXPORTED = ("lpb_default_opts", "lp_batch_create", "lp_batch_solve", "lp_batch_results",
            "lp_batch_plan_info", "lp_batch_set_timing", "lp_batch_stage_times", "lp_batch_destroy",
            "lpb_strerror", "lpb_last_error", "lp_solve_uniform_noalloc", "lp_hyperbox_solve",
            "lp_mlp_create", "lp_mlp_num_params", "lp_mlp_set_params", "lp_mlp_get_params", "lp_mlp_set_scaling",
            "lp_mlp_forward", "lp_mlp_train_step", "lp_mlp_gradients", "lp_mlp_destroy", "lp_batch_solve_warm",
            "lp_batch_features", "lp_batch_active_labels", "lp_batch_solve_graph", "lp_batch_autotune",
            "lp_batch_group_info", "lp_batch_set_group_form", "lp_solve_host", "lp_mlp_gradients_at",
            "lp_mlp_gemm_bf16", "lpb_measure_peaks", "lp_mlp_fit_scaling", "lp_mlp_get_scaling",
            "lp_mlp_tc_faults")


class LPBatchOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("max_iters", ctypes.c_int32),
        ("eps_opt", ctypes.c_double),
        ("eps_piv", ctypes.c_double),
        ("eps_feas", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("block_threads", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
    ]


class LPBatchGroup(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("count", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int64),
        ("tuned_ms", ctypes.c_float),
        ("cluster_ctas", ctypes.c_int32),
    ]


class LPBPeaks(ctypes.Structure):
    _fields_ = [
        ("fp64_gflops", ctypes.c_double),
        ("fp32_gflops", ctypes.c_double),
        ("smem_gbs", ctypes.c_double),
        ("num_sms", ctypes.c_int32),
    ]


class LPBatchPlan(ctypes.Structure):
    _fields_ = [
        ("num_groups", ctypes.c_int32),
        ("num_resident", ctypes.c_int32),
        ("num_streamed", ctypes.c_int32),
        ("num_phase1", ctypes.c_int32),
        ("num_mixed", ctypes.c_int32),
        ("num_fallback", ctypes.c_int32),
        ("internal_errors", ctypes.c_int32),
        ("internal_error_code", ctypes.c_int32),
        ("internal_error_lp", ctypes.c_int32),
        ("internal_error_detail", ctypes.c_int32 * 5),
        ("num_warm_certified", ctypes.c_int32),
        ("num_warm_rounds", ctypes.c_int32),
        ("num_cluster", ctypes.c_int32),
        ("num_warm_retried", ctypes.c_int32),
        ("max_smem_bytes", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
    ]


class LPBError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where} failed: {strerror(code)} ({detail})")


_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"CUDA solver library not built: {p} is missing "
                              "(run __graft_entry__.build() or python -m paper_1802_08557_gb300.build)")
        L = ctypes.CDLL(p)
        L.lpb_default_opts.argtypes = [ctypes.POINTER(LPBatchOpts)]
        L.lpb_default_opts.restype = None
        L.lp_batch_create.argtypes = [ctypes.POINTER(_vp), _i32, _vp, _vp,
                                      _vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _i64,
                                      _i32, ctypes.POINTER(LPBatchOpts), _vp]
        L.lp_batch_create.restype = ctypes.c_int
        L.lp_batch_solve.argtypes = [_vp, _vp]
        L.lp_batch_solve.restype = ctypes.c_int
        L.lp_batch_results.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i32]
        L.lp_batch_results.restype = ctypes.c_int
        L.lp_batch_plan_info.argtypes = [_vp, ctypes.POINTER(LPBatchPlan)]
        L.lp_batch_plan_info.restype = ctypes.c_int
        L.lp_mlp_create.argtypes = [ctypes.POINTER(_vp), _i32, _i32, _i32, _i32, _i32, ctypes.c_uint64]
        L.lp_mlp_num_params.argtypes = [_vp, ctypes.POINTER(_i64)]
        L.lp_mlp_set_params.argtypes = [_vp, _vp]
        L.lp_mlp_get_params.argtypes = [_vp, _vp]
        L.lp_mlp_set_scaling.argtypes = [_vp, _vp, _vp]
        L.lp_mlp_get_scaling.argtypes = [_vp, _vp, _vp]
        L.lp_mlp_fit_scaling.argtypes = [_vp, _vp, _i64, _vp]
        L.lp_mlp_forward.argtypes = [_vp, _vp, _i64, _vp, _vp]
        L.lp_mlp_train_step.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float,
                                        ctypes.POINTER(ctypes.c_double), _vp]
        L.lp_mlp_gradients.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, _vp, ctypes.POINTER(ctypes.c_double),
                                       _vp]
        L.lp_mlp_gradients_at.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, _vp,
                                          ctypes.POINTER(ctypes.c_double), _vp]
        L.lp_mlp_gemm_bf16.argtypes = [_i32, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _i32, _vp, _i32, _vp, _vp,
                                       _vp, _i32, _vp, _i32, _vp]
        L.lp_mlp_tc_faults.argtypes = [ctypes.POINTER(_i32)]
        L.lp_mlp_destroy.argtypes = [_vp]
        L.lp_batch_solve_graph.argtypes = [_vp, _vp]
        L.lp_batch_solve_graph.restype = ctypes.c_int
        L.lp_batch_autotune.argtypes = [_vp, _i32, _vp]
        L.lp_batch_autotune.restype = ctypes.c_int
        L.lp_batch_group_info.argtypes = [_vp, _i32, ctypes.POINTER(LPBatchGroup)]
        L.lp_batch_group_info.restype = ctypes.c_int
        L.lp_batch_set_group_form.argtypes = [_vp, _i32, _i32, _i32]
        L.lp_batch_set_group_form.restype = ctypes.c_int
        L.lp_solve_host.argtypes = [_i32, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _i64,
                                    ctypes.POINTER(LPBatchOpts), _i32, _vp, _vp, _vp, _vp, _vp]
        L.lp_solve_host.restype = ctypes.c_int
        L.lp_batch_solve_warm.argtypes = [_vp, _vp, ctypes.c_float, _vp]
        L.lp_batch_solve_warm.restype = ctypes.c_int
        L.lp_batch_features.argtypes = [_vp, _vp, _vp]
        L.lp_batch_features.restype = ctypes.c_int
        L.lp_batch_active_labels.argtypes = [_vp, _vp, _vp]
        L.lp_batch_active_labels.restype = ctypes.c_int
        for f in ("lp_mlp_create", "lp_mlp_num_params", "lp_mlp_set_params", "lp_mlp_get_params",
                  "lp_mlp_set_scaling", "lp_mlp_forward", "lp_mlp_train_step", "lp_mlp_gradients",
                  "lp_mlp_gradients_at", "lp_mlp_gemm_bf16", "lp_mlp_destroy", "lp_mlp_get_scaling",
                  "lp_mlp_fit_scaling", "lp_mlp_tc_faults"):
            getattr(L, f).restype = ctypes.c_int
        L.lp_hyperbox_solve.argtypes = [_i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _i32, _vp]
        L.lp_hyperbox_solve.restype = ctypes.c_int
        L.lp_batch_set_timing.argtypes = [_vp, _i32]
        L.lp_batch_set_timing.restype = ctypes.c_int
        L.lp_batch_stage_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_i32)]
        L.lp_batch_stage_times.restype = ctypes.c_int
        L.lp_batch_destroy.argtypes = [_vp]
        L.lp_batch_destroy.restype = ctypes.c_int
        L.lpb_strerror.argtypes = [ctypes.c_int]
        L.lpb_strerror.restype = ctypes.c_char_p
        L.lp_solve_uniform_noalloc.argtypes = [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                               ctypes.POINTER(LPBatchOpts), _vp]
        L.lp_solve_uniform_noalloc.restype = ctypes.c_int
        L.lpb_measure_peaks.argtypes = [ctypes.POINTER(LPBPeaks), _vp]
        L.lpb_measure_peaks.restype = ctypes.c_int
        L.lpb_last_error.argtypes = []
        L.lpb_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def strerror(code: int) -> str:
    try:
        return load().lpb_strerror(code).decode()
    except ImportError:
        return f"error {code}"


def _check(code: int, where: str):
    if code != LPB_OK:
        raise LPBError(code, where, load().lpb_last_error().decode())


def lpb_default_opts(**overrides) -> LPBatchOpts:
    o = LPBatchOpts()
    load().lpb_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _addr(a) -> int | None:
    """Address of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def lp_batch_create(m, n, a_off, A, b_off, b, c_off, c, ptr_kind: int, opts: LPBatchOpts | None = None,
                    stream=None):
    """Returns an opaque handle (c_void_p).  ``m, n, *_off`` are numpy arrays
    (host); A, b, c are numpy arrays (LPB_HOST) or CUDA tensors (LPB_DEVICE)."""
    L = load()
    m = np.ascontiguousarray(m, np.int32)
    n = np.ascontiguousarray(n, np.int32)
    a_off = None if a_off is None else np.ascontiguousarray(a_off, np.int64)
    b_off = None if b_off is None else np.ascontiguousarray(b_off, np.int64)
    c_off = None if c_off is None else np.ascontiguousarray(c_off, np.int64)
    h = _vp()
    lens = [int(np.prod(np.shape(v))) if isinstance(v, np.ndarray) else int(v.numel()) for v in (A, b, c)]
    code = L.lp_batch_create(ctypes.byref(h), int(m.shape[0]), _addr(m), _addr(n),
                             _addr(a_off), _addr(A), lens[0], _addr(b_off), _addr(b), lens[1],
                             _addr(c_off), _addr(c), lens[2], ptr_kind,
                             ctypes.byref(opts) if opts is not None else None, _stream_handle(stream))
    _check(code, "lp_batch_create")
    return h


def lp_solve_host(m, n, a_off, A, b_off, b, c_off, c, status, iters, obj, x, y=None,
                  opts: LPBatchOpts | None = None, chunks: int = 0):
    """One call from host arrays (numpy or pinned CPU tensors) to host result
    arrays, the input copies overlapped with the solve (see include/lpbatch.h)."""
    L = load()
    m = np.ascontiguousarray(m, np.int32)
    n = np.ascontiguousarray(n, np.int32)
    a_off = None if a_off is None else np.ascontiguousarray(a_off, np.int64)
    b_off = None if b_off is None else np.ascontiguousarray(b_off, np.int64)
    c_off = None if c_off is None else np.ascontiguousarray(c_off, np.int64)
    lens = [int(np.prod(np.shape(v))) if isinstance(v, np.ndarray) else int(v.numel()) for v in (A, b, c)]
    code = L.lp_solve_host(int(m.shape[0]), _addr(m), _addr(n), _addr(a_off), _addr(A), lens[0],
                           _addr(b_off), _addr(b), lens[1], _addr(c_off), _addr(c), lens[2],
                           ctypes.byref(opts) if opts is not None else None, int(chunks),
                           _addr(status), _addr(iters), _addr(obj), _addr(x), _addr(y))
    _check(code, "lp_solve_host")


def lp_batch_solve(h, stream=None):
    _check(load().lp_batch_solve(h, _stream_handle(stream)), "lp_batch_solve")


def lp_batch_results(h, status=None, iters=None, obj=None, x=None, y=None, ptr_kind: int = LPB_HOST):
    _check(load().lp_batch_results(h, _addr(status), _addr(iters), _addr(obj), _addr(x), _addr(y), ptr_kind),
           "lp_batch_results")


def lp_batch_plan_info(h) -> dict:
    p = LPBatchPlan()
    _check(load().lp_batch_plan_info(h, ctypes.byref(p)), "lp_batch_plan_info")
    out = {name: getattr(p, name) for name, _ in LPBatchPlan._fields_}
    out["internal_error_detail"] = list(out["internal_error_detail"])
    return out


def lp_batch_set_timing(h, enable: bool = True):
    _check(load().lp_batch_set_timing(h, 1 if enable else 0), "lp_batch_set_timing")


def lp_batch_stage_times(h):
    """(mean ms of all launch groups, mean ms of the FP64 re-solve, solves
    covered) since timing was enabled or last read."""
    ms = (ctypes.c_float * 2)()
    n = _i32(0)
    _check(load().lp_batch_stage_times(h, ms, ctypes.byref(n)), "lp_batch_stage_times")
    return float(ms[0]), float(ms[1]), int(n.value)


def lp_hyperbox_solve(L, lo, hi, obj, x=None, box_per_lp: bool = False, ptr_kind: int = LPB_HOST, stream=None):
    """Eq. 7 for every row of ``L`` (num_lps x dim): obj[k] = max of L[k].x
    over the box, x[k] the maximiser (see include/lpbatch.h).  Arrays are
    numpy (LPB_HOST) or CUDA tensors (LPB_DEVICE), C-contiguous float64."""
    num_lps, dim = (int(L.shape[0]), int(L.shape[1])) if len(L.shape) == 2 else (0, 0)
    _check(load().lp_hyperbox_solve(num_lps, dim, _addr(lo), _addr(hi), 1 if box_per_lp else 0, _addr(L),
                                    _addr(obj), _addr(x), ptr_kind, _stream_handle(stream)), "lp_hyperbox_solve")


class Mlp:
    """Owner of one warm-start network handle (see include/lpbatch.h)."""

    def __init__(self, n_in: int, n_h1: int, n_h2: int, n_out: int, max_batch: int, seed: int = 0):
        self.sizes = (n_in, n_h1, n_h2, n_out)
        self.h = _vp()
        _check(load().lp_mlp_create(ctypes.byref(self.h), n_in, n_h1, n_h2, n_out, max_batch, seed),
               "lp_mlp_create")
        n = _i64(0)
        _check(load().lp_mlp_num_params(self.h, ctypes.byref(n)), "lp_mlp_num_params")
        self.num_params = int(n.value)

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params, np.float32)
        _check(load().lp_mlp_get_params(self.h, p.ctypes.data), "lp_mlp_get_params")
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.num_params
        _check(load().lp_mlp_set_params(self.h, p.ctypes.data), "lp_mlp_set_params")

    def set_scaling(self, mean: np.ndarray, inv_std: np.ndarray):
        mean = np.ascontiguousarray(mean, np.float32)
        inv_std = np.ascontiguousarray(inv_std, np.float32)
        _check(load().lp_mlp_set_scaling(self.h, mean.ctypes.data, inv_std.ctypes.data), "lp_mlp_set_scaling")

    def get_scaling(self):
        mean = np.empty(self.sizes[0], np.float32)
        inv = np.empty(self.sizes[0], np.float32)
        _check(load().lp_mlp_get_scaling(self.h, mean.ctypes.data, inv.ctypes.data), "lp_mlp_get_scaling")
        return mean, inv

    def fit_scaling(self, x, stream=None):
        """Input scaling from device features x [rows x n_in] (FP32)."""
        _check(load().lp_mlp_fit_scaling(self.h, _addr(x), int(x.shape[0]), _stream_handle(stream)),
               "lp_mlp_fit_scaling")

    def forward(self, x, logits, stream=None):
        _check(load().lp_mlp_forward(self.h, _addr(x), int(x.shape[0]), _addr(logits), _stream_handle(stream)),
               "lp_mlp_forward")

    def train_step(self, x, y, lr: float, pos_weight: float = 1.0, want_loss: bool = False, stream=None):
        loss = ctypes.c_double(0.0)
        _check(load().lp_mlp_train_step(self.h, _addr(x), _addr(y), int(x.shape[0]), lr, pos_weight,
                                        ctypes.byref(loss) if want_loss else None, _stream_handle(stream)),
               "lp_mlp_train_step")
        return loss.value if want_loss else None

    def gradients(self, x, y, pos_weight: float = 1.0, stream=None):
        g = np.empty(self.num_params, np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().lp_mlp_gradients(self.h, _addr(x), _addr(y), int(x.shape[0]), pos_weight, g.ctypes.data,
                                       ctypes.byref(loss), _stream_handle(stream)), "lp_mlp_gradients")
        return g, loss.value

    def gradients_at(self, x, a1, a2, z, y, pos_weight: float = 1.0, stream=None):
        """Gradients from given forward values a1, a2, z (device FP32)."""
        g = np.empty(self.num_params, np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().lp_mlp_gradients_at(self.h, _addr(x), _addr(a1), _addr(a2), _addr(z), _addr(y),
                                          int(x.shape[0]), pos_weight, g.ctypes.data, ctypes.byref(loss),
                                          _stream_handle(stream)), "lp_mlp_gradients_at")
        return g, loss.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().lp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lp_mlp_tc_faults() -> int:
    """Tiles of the tcgen05 product kernel that gave up on a wait (0 normally)."""
    c = _i32(0)
    _check(load().lp_mlp_tc_faults(ctypes.byref(c)), "lp_mlp_tc_faults")
    return int(c.value)


def lpb_measure_peaks(stream=None) -> dict:
    """Measured FP64/FP32 FMA and shared-memory throughputs of the device."""
    p = LPBPeaks()
    _check(load().lpb_measure_peaks(ctypes.byref(p), _stream_handle(stream)), "lpb_measure_peaks")
    return {"fp64_gflops": p.fp64_gflops, "fp32_gflops": p.fp32_gflops, "smem_gbs": p.smem_gbs,
            "num_sms": p.num_sms}


def lp_mlp_gemm_bf16(epilogue, form, M, N, K, A, lda, B, ldb, C=None, ldc=0, bias=None, pre=None, h=None, ldh=0,
                     hT=None, ldt=0, stream=None):
    """The network's product kernel on caller device buffers (see
    include/lpbatch.h); A, B, h, hT are BF16 tensors (torch.bfloat16)."""
    _check(load().lp_mlp_gemm_bf16(int(epilogue), int(form), int(M), int(N), int(K), _addr(A), int(lda), _addr(B),
                                   int(ldb), _addr(C), int(ldc), _addr(bias), _addr(pre), _addr(h), int(ldh),
                                   _addr(hT), int(ldt), _stream_handle(stream)), "lp_mlp_gemm_bf16")


def lp_solve_uniform_noalloc(num_lps, m, n, A, b, c, status, iters, obj, x, y=None,
                             opts: LPBatchOpts | None = None, stream=None) -> int:
    """Solve equal-size LPs with caller-owned device buffers and no allocation
    (see include/lpbatch.h).  Returns the lpb_err code (no message is
    recorded by this entry point)."""
    return load().lp_solve_uniform_noalloc(int(num_lps), int(m), int(n), _addr(A), _addr(b), _addr(c),
                                           _addr(status), _addr(iters), _addr(obj), _addr(x), _addr(y),
                                           ctypes.byref(opts) if opts is not None else None,
                                           _stream_handle(stream))


def lp_batch_solve_graph(h, stream=None):
    _check(load().lp_batch_solve_graph(h, _stream_handle(stream)), "lp_batch_solve_graph")


def lp_batch_autotune(h, rounds: int = 2, stream=None):
    _check(load().lp_batch_autotune(h, rounds, _stream_handle(stream)), "lp_batch_autotune")


def lp_batch_groups(h) -> list:
    """The plan's launch groups as dicts (see include/lpbatch.h)."""
    out = []
    n = lp_batch_plan_info(h)["num_groups"]
    for i in range(n):
        g = LPBatchGroup()
        if load().lp_batch_group_info(h, i, ctypes.byref(g)) != LPB_OK:
            break
        out.append({name: getattr(g, name) for name, _ in LPBatchGroup._fields_})
    return out


def lp_batch_set_group_form(h, index: int, threads: int, persistent: bool):
    _check(load().lp_batch_set_group_form(h, index, threads, 1 if persistent else 0), "lp_batch_set_group_form")


def lp_batch_solve_warm(h, net, threshold: float = 0.2, stream=None):
    """Warm solve from the network's proposal (see include/lpbatch.h)."""
    _check(load().lp_batch_solve_warm(h, net.h, threshold, _stream_handle(stream)), "lp_batch_solve_warm")


def lp_batch_features(h, x, stream=None):
    _check(load().lp_batch_features(h, _addr(x), _stream_handle(stream)), "lp_batch_features")


def lp_batch_active_labels(h, labels, stream=None):
    _check(load().lp_batch_active_labels(h, _addr(labels), _stream_handle(stream)), "lp_batch_active_labels")


def lp_batch_destroy(h):
    _check(load().lp_batch_destroy(h), "lp_batch_destroy")


class BatchSolver:
    """Convenience owner of one batch handle (``workloads.LPBatch`` input)."""

    def __init__(self, batch, device_data: bool = True, opts: LPBatchOpts | None = None, stream=None):
        self.batch = batch
        self.num_lps = batch.num_lps
        self.total_x = int(batch.n.astype(np.int64).sum())
        self.total_y = int(batch.m.astype(np.int64).sum())
        if device_data:
            import torch
            A = torch.from_numpy(batch.A).cuda()
            b = torch.from_numpy(batch.b).cuda()
            c = torch.from_numpy(batch.c).cuda()
            torch.cuda.synchronize()
            self.h = lp_batch_create(batch.m, batch.n, batch.a_off, A, batch.b_off, b, batch.c_off, c,
                                     LPB_DEVICE, opts, stream)
            del A, b, c
        else:
            self.h = lp_batch_create(batch.m, batch.n, batch.a_off, batch.A, batch.b_off, batch.b,
                                     batch.c_off, batch.c, LPB_HOST, opts, stream)

    def solve(self, stream=None):
        lp_batch_solve(self.h, stream)

    def results(self):
        status = np.zeros(self.num_lps, np.int32)
        iters = np.zeros(self.num_lps, np.int32)
        obj = np.zeros(self.num_lps)
        x = np.zeros(self.total_x)
        y = np.zeros(self.total_y)
        lp_batch_results(self.h, status, iters, obj, x, y, LPB_HOST)
        return dict(status=status, iters=iters, obj=obj, x=x, y=y)

    def plan_info(self):
        return lp_batch_plan_info(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            lp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
