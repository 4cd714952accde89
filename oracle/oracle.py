"""ctypes binding of the plain-C FP64 oracle (test infrastructure only).

Every function takes and returns numpy arrays; matrices are row-major
float64, the layout the GPU library also uses.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lu_oracle.c")
_DEPS = [_SRC, os.path.join(_HERE, "lu_oracle_body.h")]
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"liblu_oracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile lu_oracle.c with gcc (-ffp-contract=off keeps every fused
    operation explicit).  Returns the shared-library path."""
    out = lib_path()
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in _DEPS):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Counts(ctypes.Structure):
    _fields_ = [("s1_div", ctypes.c_longlong), ("s2_fma", ctypes.c_longlong)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_lu_factor.argtypes = [I, I, P, I, I, I, P, P, P]
            lib.oracle_lu_factor.restype = I
            lib.oracle_tslu_select.argtypes = [I, I, P, I, I, I, P]
            lib.oracle_tslu_select.restype = I
            lib.oracle_lu_solve.argtypes = [I, I, P, I, P, P, I]
            lib.oracle_lu_solve.restype = I
            lib.oracle_backward_error.argtypes = [I, I, P, I, P, I, P, I, P]
            lib.oracle_backward_error.restype = None
            lib.oracle_set_threads.argtypes = [I]
            lib.oracle_set_threads.restype = I
            lib.oracle_lu_factor_f32.argtypes = [I, I, P, I, I, I, P, P, P]
            lib.oracle_lu_factor_f32.restype = I
            lib.oracle_lu_factor_q_f32.argtypes = [I, I, P, I, I, I, P, P, P, I]
            lib.oracle_lu_factor_q_f32.restype = I
            lib.oracle_lu_solve_f32.argtypes = [I, I, P, I, P, P, I]
            lib.oracle_lu_solve_f32.restype = I
            lib.oracle_gemm_lowp.argtypes = [I, I, I, P, I, P, I, P, I, I, P, P]
            lib.oracle_gemm_lowp.restype = None
            lib.oracle_round_array.argtypes = [P, P, ctypes.c_longlong, I]
            lib.oracle_round_array.restype = None
            for suf in ("", "_f32"):
                getattr(lib, "oracle_chol_factor" + suf).argtypes = [I, P, I, P]
                getattr(lib, "oracle_chol_factor" + suf).restype = I
                getattr(lib, "oracle_chol_solve" + suf).argtypes = [I, I, P, I, P, I]
                getattr(lib, "oracle_chol_solve" + suf).restype = I
            lib.oracle_e4m3_exponent.argtypes = [ctypes.c_float]
            lib.oracle_e4m3_exponent.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count used."""
    return _load().oracle_set_threads(int(n))


def lu_factor(A: np.ndarray, b: int, h: int = 128, count: bool = False):
    """Tournament-pivoting LU of an m x n matrix.

    Returns (LU, piv, info) or (LU, piv, info, (s1_div, s2_fma)) when
    ``count``; LU is a new array, piv is 0-based LAPACK-style (int32)."""
    lib = _load()
    LU = np.ascontiguousarray(A, dtype=np.float64).copy()
    m, n = LU.shape
    piv = np.zeros(max(min(m, n), 1), dtype=np.int32)
    info = ctypes.c_int(0)
    cnt = _Counts()
    rc = lib.oracle_lu_factor(m, n, _ptr(LU), max(n, 1), int(b), int(h), _ptr(piv),
                              ctypes.byref(info), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError(f"oracle_lu_factor: argument {-rc} invalid")
    piv = piv[: min(m, n)]
    if count:
        return LU, piv, info.value, (cnt.s1_div, cnt.s2_fma)
    return LU, piv, info.value


def tslu_select(A: np.ndarray, k: int, w: int, h: int) -> np.ndarray:
    """Winners (row positions, root pivot order) of one TournPivot on panel
    columns [k, k+w) over active rows [k, m) of A's current values."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    win = np.zeros(w, dtype=np.int32)
    rc = lib.oracle_tslu_select(m, max(n, 1), _ptr(A), int(k), int(w), int(h), _ptr(win))
    if rc != 0:
        raise ValueError("oracle_tslu_select: bad arguments")
    return win


def lu_solve(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = U^{-1} L^{-1} P B for the oracle's factors; B is n or n x nrhs."""
    lib = _load()
    LU = np.ascontiguousarray(LU, dtype=np.float64)
    n = LU.shape[0]
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(n, -1), dtype=np.float64).copy()
    nrhs = X.shape[1]
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    rc = lib.oracle_lu_solve(n, nrhs, _ptr(LU), max(n, 1), _ptr(piv), _ptr(X), max(nrhs, 1))
    if rc != 0:
        raise ValueError(f"oracle_lu_solve: argument {-rc} invalid")
    return X[:, 0] if vec else X


def backward_error(A: np.ndarray, B: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Per-column normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    Bm = np.ascontiguousarray(B.reshape(n, -1), dtype=np.float64)
    Xm = np.ascontiguousarray(X.reshape(n, -1), dtype=np.float64)
    nrhs = Bm.shape[1]
    eta = np.zeros(nrhs, dtype=np.float64)
    lib.oracle_backward_error(n, nrhs, _ptr(A), max(n, 1), _ptr(Bm), max(nrhs, 1),
                              _ptr(Xm), max(nrhs, 1), _ptr(eta))
    return eta


def lu_factor_f32(A: np.ndarray, b: int, h: int = 128, lowp: int = 0):
    """binary32 instance of the same tournament LU (fmaf, IEEE float division).
    lowp = 1 / 2: the Schur update takes bfloat16 / fp8-e4m3 operands with
    per-256-block power-of-two scales (the mixed-precision factorization)."""
    lib = _load()
    LU = np.ascontiguousarray(A, dtype=np.float32).copy()
    m, n = LU.shape
    piv = np.zeros(max(min(m, n), 1), dtype=np.int32)
    info = ctypes.c_int(0)
    cnt = _Counts()
    rc = lib.oracle_lu_factor_q_f32(m, n, _ptr(LU), max(n, 1), int(b), int(h), _ptr(piv),
                                    ctypes.byref(info), ctypes.byref(cnt), int(lowp))
    if rc != 0:
        raise ValueError(f"oracle_lu_factor_f32: argument {-rc} invalid")
    return LU, piv[: min(m, n)], info.value


def lu_solve_f32(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    lib = _load()
    LU = np.ascontiguousarray(LU, dtype=np.float32)
    n = LU.shape[0]
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(n, -1), dtype=np.float32).copy()
    nrhs = X.shape[1]
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    lib.oracle_lu_solve_f32(n, nrhs, _ptr(LU), max(n, 1), _ptr(piv), _ptr(X), max(nrhs, 1))
    return X[:, 0] if vec else X


def round_lowp(x: np.ndarray, fp8: bool) -> np.ndarray:
    """bfloat16 (fp8=False) or fp8 e4m3 with saturation (fp8=True), as float32."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib.oracle_round_array(_ptr(x), _ptr(y), x.size, 1 if fp8 else 0)
    return y


def e4m3_exponent(maxabs: float) -> int:
    return _load().oracle_e4m3_exponent(float(maxabs))


def gemm_lowp(L: np.ndarray, U: np.ndarray, C: np.ndarray, fp8: bool):
    """Reference of C - s * q(L) q(U) with per-256-block power-of-two scales.
    Returns (Cref, Sabs) in float64 (Sabs = s * sum |qL qU|)."""
    lib = _load()
    L = np.ascontiguousarray(L, dtype=np.float32)
    U = np.ascontiguousarray(U, dtype=np.float32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    M, K = L.shape
    K2, N = U.shape
    assert K == K2 and C.shape == (M, N)
    Cref = np.empty((M, N), dtype=np.float64)
    Sabs = np.empty((M, N), dtype=np.float64)
    lib.oracle_gemm_lowp(M, N, K, _ptr(L), max(K, 1), _ptr(U), max(N, 1), _ptr(C), max(N, 1),
                         1 if fp8 else 0, _ptr(Cref), _ptr(Sabs))
    return Cref, Sabs


def chol_factor(A: np.ndarray, dtype=np.float64):
    """Cholesky A = L L^T (lower triangle read and written, strict upper
    untouched).  Returns (F, info): F is a new array whose lower triangle is
    L (columns before info - 1 when info > 0); dtype float64 or float32
    selects the binary64 or binary32 instance."""
    lib = _load()
    F = np.ascontiguousarray(A, dtype=dtype).copy()
    n = F.shape[0]
    assert F.shape == (n, n)
    info = ctypes.c_int(0)
    fn = lib.oracle_chol_factor if F.dtype == np.float64 else lib.oracle_chol_factor_f32
    rc = fn(n, _ptr(F), max(n, 1), ctypes.byref(info))
    if rc != 0:
        raise ValueError(f"oracle_chol_factor: argument {-rc} invalid")
    return F, info.value


def chol_solve(F: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = L^{-T} L^{-1} B with L the lower triangle of F; B is n or n x nrhs.
    The precision is F's (float64 or float32)."""
    lib = _load()
    F = np.ascontiguousarray(F)
    n = F.shape[0]
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(n, -1), dtype=F.dtype).copy()
    nrhs = X.shape[1]
    fn = lib.oracle_chol_solve if F.dtype == np.float64 else lib.oracle_chol_solve_f32
    rc = fn(n, nrhs, _ptr(F), max(n, 1), _ptr(X), max(nrhs, 1))
    if rc != 0:
        raise ValueError(f"oracle_chol_solve: argument {-rc} invalid")
    return X[:, 0] if vec else X
