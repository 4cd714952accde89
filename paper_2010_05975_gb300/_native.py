"""ctypes loader for the in-tree CUDA library (no fallback of any kind)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LU_ENOMEM = 1
LU_ELAUNCH = 2
LU_ETIMEOUT = 3
LU_EBUSY = 4
LU_EUNSUPPORTED = 5
LU_ENOTFOUND = 6

LU_WAIT_SITE_TC = 0
LU_WAIT_SITE_SOLVE = 1

LU_PREC_F64 = 0
LU_PREC_F32 = 1
LU_PREC_BF16 = 2
LU_PREC_FP8 = 3

_NAMES = {LU_ENOMEM: "LU_ENOMEM", LU_ELAUNCH: "LU_ELAUNCH", LU_ETIMEOUT: "LU_ETIMEOUT",
          LU_EBUSY: "LU_EBUSY", LU_EUNSUPPORTED: "LU_EUNSUPPORTED", LU_ENOTFOUND: "LU_ENOTFOUND"}


class LuError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        what = f"argument {-code} invalid" if code < 0 else _NAMES.get(code, f"error {code}")
        super().__init__(f"{fn}: {what}")


class lu_opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("h", ctypes.c_int), ("precision", ctypes.c_int), ("defer", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class ir_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("b", ctypes.c_int), ("h", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("krylov_products", ctypes.c_int),
                ("inner_steps", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class ir_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("gmres_iters", ctypes.c_int), ("path", ctypes.c_int),
                ("info", ctypes.c_int), ("eta", ctypes.c_double), ("eta0", ctypes.c_double),
                ("precision", ctypes.c_int), ("refactors", ctypes.c_int), ("cycles32", ctypes.c_int),
                ("cycles64", ctypes.c_int), ("inner_steps", ctypes.c_int)]


class serve_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_queue", ctypes.c_int), ("dry_run", ctypes.c_int),
                ("batch_n_max", ctypes.c_int), ("batch_max", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class serve_req(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nrhs", ctypes.c_int), ("A", ctypes.c_void_p), ("lda", ctypes.c_int),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int), ("device_inputs", ctypes.c_int),
                ("matrix_id", ctypes.c_uint64), ("tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("flags", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class serve_status(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("error", ctypes.c_int), ("eta", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double), ("iters", ctypes.c_int),
                ("gmres_iters", ctypes.c_int), ("path", ctypes.c_int), ("precision", ctypes.c_int),
                ("cache_hit", ctypes.c_int), ("batched", ctypes.c_int)]


class serve_stats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("queued", ctypes.c_int), ("running", ctypes.c_int), ("peak_running", ctypes.c_int),
                ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("cache_hits", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("cache_entries", ctypes.c_int),
                ("batches", ctypes.c_longlong), ("batched", ctypes.c_longlong)]


SERVE_PENDING, SERVE_RUNNING, SERVE_DONE, SERVE_FAILED = 0, 1, 2, 3
SERVE_FLAG_FAIL = 1
SERVE_FLAG_BORROW = 2


class lu_prof_entry(ctypes.Structure):
    _fields_ = [("kernel_class", ctypes.c_int), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("total_flops", ctypes.c_double), ("total_bytes", ctypes.c_double)]


PROF_CLASSES = ["tslu", "pivot", "trsm_l21", "trsm_u12", "schur_f64", "schur_lowp", "solve", "residual", "other",
                "chol_diag", "syrk", "matvec32"]

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int

# name -> (argtypes, restype)
_SIGS = {
    "lu_factor": ([I, P, I, P, P, P], I),
    "lu_factor_ex": ([I, I, P, I, P, P, ctypes.POINTER(lu_opts), P], I),
    "lu_factor_host": ([I, I, P, I, P, P, ctypes.POINTER(lu_opts), P], I),
    "lu_solve": ([I, I, P, I, P, P, I, P], I),
    "lu_factor_f32": ([I, I, P, I, P, P, ctypes.POINTER(lu_opts), P], I),
    "lu_solve_f32": ([I, I, P, I, P, P, I, P], I),
    "lu_gemm_lowp": ([I, I, I, P, I, P, I, P, I, I, P, P], I),
    "chol_factor": ([I, P, I, P, ctypes.POINTER(lu_opts), P], I),
    "chol_factor_f32": ([I, P, I, P, ctypes.POINTER(lu_opts), P], I),
    "chol_solve": ([I, I, P, I, P, I, P], I),
    "chol_solve_f32": ([I, I, P, I, P, I, P], I),
    "lu_residual": ([I, I, P, I, P, I, P, I, P, I, P, P], I),
    "lu_memory_pool": ([ctypes.POINTER(ctypes.c_void_p)], I),
    "ir_solve": ([I, I, P, I, P, I, P, I, ctypes.POINTER(ir_opts), ctypes.POINTER(ir_result), P], I),
    "lu_factor_batched": ([I, P, P, P, P, P, I, P], I),
    "lu_solve_batched": ([I, P, P, P, P, P, P, P, I, P], I),
    "lu_batched_panel_width": ([I], I),
    "lu_batched_panel_width_dt": ([I, I], I),
    "lu_batched_set_panel_widths": ([I, P, I], I),
    "lu_residual_noalloc": ([I, I, P, I, P, I, P, I, P, I, P, P], I),
    "serve_create": ([ctypes.POINTER(serve_cfg), ctypes.POINTER(P)], I),
    "serve_enqueue": ([P, ctypes.POINTER(serve_req), ctypes.POINTER(ctypes.c_uint64)], I),
    "serve_poll": ([P, ctypes.c_uint64, ctypes.POINTER(serve_status), P], I),
    "serve_get_stats": ([P, ctypes.POINTER(serve_stats)], I),
    "serve_destroy": ([P], I),
    "lu_prof_begin": ([], I),
    "lu_prof_end": ([P, I, P], I),
    "lu_kernel_launch_count": ([], ctypes.c_ulonglong),
    "lu_test_wait_config": ([I, ctypes.c_longlong, I], I),
    "lu_wait_deadline_ns": ([I], ctypes.c_longlong),
}


def library_path() -> str:
    return _build.lib_path()


def library(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the shared library.  Raises if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path) or not _build.up_to_date():
                if not build_if_missing:
                    raise RuntimeError(
                        f"CUDA library {path} is missing or stale; build it with "
                        "paper_2010_05975_gb300.build.build() (nvcc, sm_103a)")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def register(name: str, argtypes, restype=ctypes.c_int):
    _SIGS[name] = (argtypes, restype)
    if _lib is not None and hasattr(_lib, name):
        fn = getattr(_lib, name)
        fn.argtypes = argtypes
        fn.restype = restype


def exported_symbols(lib: ctypes.CDLL, names) -> dict:
    return {n: hasattr(lib, n) for n in names}


def check(fn: str, rc: int) -> None:
    if rc != 0:
        raise LuError(fn, rc)
