"""Python face of the C ABI: same names, torch tensors in, raw pointers out."""
from __future__ import annotations

import ctypes

import torch

from . import _native as nat


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require(t: torch.Tensor, name: str, dtype, ndim: int):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    if ndim == 2 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major with unit column stride")


def lu_factor(A: torch.Tensor, piv: torch.Tensor | None = None, info: torch.Tensor | None = None,
              stream=None):
    """In-place PA = LU of a square float64 CUDA tensor.  Returns (piv, info)
    as int32 CUDA tensors (piv 0-based LAPACK style); nothing is synchronised."""
    _require(A, "A", torch.float64, 2)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("lu_factor needs a square matrix; use lu_factor_ex")
    if piv is None:
        piv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    lib = nat.library()
    rc = lib.lu_factor(n, A.data_ptr(), max(A.stride(0), 1), piv.data_ptr(), info.data_ptr(),
                       _stream_handle(stream))
    nat.check("lu_factor", rc)
    return piv[:n], info


def lu_factor_ex(A: torch.Tensor, b: int = 0, h: int = 0, precision: int = nat.LU_PREC_F64,
                 piv: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None):
    """In-place m x n factorization with panel width b and leaf height h."""
    _require(A, "A", torch.float64, 2)
    m, n = A.shape
    k = min(m, n)
    if piv is None:
        piv = torch.empty(max(k, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    opts = nat.lu_opts(b, h, precision)
    lib = nat.library()
    rc = lib.lu_factor_ex(m, n, A.data_ptr(), max(A.stride(0), 1), piv.data_ptr(), info.data_ptr(),
                          ctypes.byref(opts), _stream_handle(stream))
    nat.check("lu_factor_ex", rc)
    return piv[:k], info


def lu_solve(LU: torch.Tensor, piv: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """Overwrite B (n or n x nrhs, float64, CUDA) with the solution of A X = B."""
    _require(LU, "LU", torch.float64, 2)
    n = LU.shape[0]
    B2 = B if B.dim() == 2 else B.view(n, 1)
    _require(B2, "B", torch.float64, 2)
    lib = nat.library()
    rc = lib.lu_solve(n, B2.shape[1], LU.data_ptr(), max(LU.stride(0), 1), piv.data_ptr(), B2.data_ptr(),
                      max(B2.stride(0), 1), _stream_handle(stream))
    nat.check("lu_solve", rc)
    return B
