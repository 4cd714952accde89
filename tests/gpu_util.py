"""Helpers for the GPU parity tests (device placement, host copies)."""
from __future__ import annotations

import numpy as np
import pytest


def cuda_or_fail():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA (run with -m 'not gpu' here)")
    return torch


def lib():
    import paper_2010_05975_gb300 as g
    from paper_2010_05975_gb300 import build
    build.build()
    return g


def to_dev(A: np.ndarray, lda: int | None = None):
    """Row-major float64 device copy, optionally with a padded leading dimension."""
    torch = cuda_or_fail()
    m, n = A.shape
    if lda is None or lda == n:
        return torch.from_numpy(np.ascontiguousarray(A)).cuda(), None
    buf = torch.full((m, lda), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    return buf[:, :n], buf


def split_lu(LU):
    m, n = LU.shape
    k = min(m, n)
    L = np.tril(LU[:, :k], -1) + np.eye(m, k)
    U = np.triu(LU[:k, :])
    return L, U


def apply_piv(A, piv):
    PA = np.array(A, copy=True)
    for i, p in enumerate(piv):
        if p != i:
            PA[[i, p]] = PA[[p, i]]
    return PA


def factor_close(X, R, tol=1e-10):
    """Reading of 'within 1e-10 relative': |x - r| <= tol * max(|r|, max|row of r|)."""
    scale = np.maximum(np.abs(R), np.abs(R).max(axis=1, keepdims=True))
    bad = np.abs(X - R) > tol * np.maximum(scale, 1e-300)
    return not bad.any(), int(bad.sum())
