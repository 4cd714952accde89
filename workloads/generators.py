"""Counter-based seeded generators (splitmix64) for the synthetic workloads.

Every value is a pure function of (seed, stream, index), so any slice of a
matrix can be regenerated independently and the same array feeds both the
oracle and the GPU path.  splitmix64 is Steele, Lea and Flood's finaliser
(the increment 0x9E3779B97F4A7C15 and the two multiply-xorshift rounds of
its published definition).

Workloads:
  * uniform entries in [-1, 1)                    (N=512 single matrix, batches)
  * N(0, 1) entries via Box-Muller                (N=32768 single matrix)
  * A = H1 diag(s) H2 with Householder products   (mixed precision + refinement)
  * symmetric, uniform entries + n on the diagonal (Cholesky)
  * log-uniform sizes, Poisson arrival times      (batches, serving)
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """64-bit hash of counter ``idx`` (uint64 array) under key (seed, stream)."""
    key = np.uint64(((int(seed) & 0xFFFFFFFF) << 32 | (int(stream) & 0xFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (key * _GOLDEN) ^ ((idx.astype(np.uint64) + np.uint64(1)) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of the hash times 2^-53."""
    return (splitmix64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [-1, 1) (2u - 1 is exact in binary64)."""
    return 2.0 * uniform01(seed, stream, idx) - 1.0


def normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """N(0, 1) via Box-Muller on two independent uniforms of the same counter."""
    u1 = 1.0 - uniform01(seed, 2 * stream, idx)          # (0, 1]
    u2 = uniform01(seed, 2 * stream + 1, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _fill(m: int, n: int, fn, seed: int, stream: int, out: np.ndarray | None, threads: int | None):
    A = np.empty((m, n), dtype=np.float64) if out is None else out
    rows_per = max(1, (1 << 22) // max(n, 1))
    chunks = [(r, min(m, r + rows_per)) for r in range(0, m, rows_per)]

    def work(c):
        r0, r1 = c
        idx = np.arange(r0 * n, r1 * n, dtype=np.uint64)
        A[r0:r1, :] = fn(seed, stream, idx).reshape(r1 - r0, n)

    nt = threads or min(32, os.cpu_count() or 1)
    if len(chunks) == 1 or nt == 1:
        for c in chunks:
            work(c)
    else:
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, chunks))
    return A


def matrix_uniform(m: int, n: int, seed: int, stream: int = 0, shift: float = 0.0,
                   out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """m x n row-major matrix, entries iid Uniform[-1, 1), plus shift*I."""
    A = _fill(m, n, uniform_pm1, seed, stream, out, threads)
    if shift != 0.0:
        d = np.arange(min(m, n))
        A[d, d] += shift
    return A


def matrix_normal(m: int, n: int, seed: int, stream: int = 0,
                  out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """m x n row-major matrix, entries iid N(0, 1)."""
    return _fill(m, n, normal, seed, stream, out, threads)


def matrix_spd(n: int, seed: int, stream: int = 0, shift: float | None = None,
               out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """n x n symmetric matrix: a_ij = a_ji = Uniform[-1, 1) drawn at counter
    min(i,j) * n + max(i,j), plus shift on the diagonal (default n, which
    makes it strictly diagonally dominant with a positive diagonal, hence
    positive definite; a small shift gives an indefinite matrix)."""
    A = np.empty((n, n), dtype=np.float64) if out is None else out
    rows_per = max(1, (1 << 22) // max(n, 1))
    chunks = [(r, min(n, r + rows_per)) for r in range(0, n, rows_per)]
    cols = np.arange(n, dtype=np.uint64)

    def work(c):
        r0, r1 = c
        i = np.arange(r0, r1, dtype=np.uint64)[:, None]
        lo = np.minimum(i, cols[None, :])
        hi = np.maximum(i, cols[None, :])
        A[r0:r1, :] = uniform_pm1(seed, stream, (lo * np.uint64(n) + hi).ravel()).reshape(r1 - r0, n)

    nt = threads or min(32, os.cpu_count() or 1)
    if len(chunks) == 1 or nt == 1:
        for c in chunks:
            work(c)
    else:
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, chunks))
    d = np.arange(n)
    A[d, d] += float(n) if shift is None else shift
    return A


def _reflectors(n: int, count: int, seed: int, stream: int) -> np.ndarray:
    V = np.empty((count, n), dtype=np.float64)
    for r in range(count):
        V[r] = normal(seed, stream * 64 + r, np.arange(n, dtype=np.uint64))
        V[r] /= np.linalg.norm(V[r])
    return V


def householder_diag(n: int, kappa: float, seed: int, count: int = 8):
    """A = H1 diag(s) H2 with H1, H2 products of ``count`` seeded Householder
    reflectors (I - 2 v v^T, |v| = 1) and s_i = kappa^(-i/(n-1)), so the
    2-norm condition number is kappa and A^{-1} = H2^T diag(1/s) H1^T.

    Returns (A, V1, V2, s) where V1, V2 hold the unit reflector vectors."""
    V1 = _reflectors(n, count, seed, 1)
    V2 = _reflectors(n, count, seed, 2)
    s = kappa ** (-np.arange(n, dtype=np.float64) / max(n - 1, 1))
    A = np.zeros((n, n), dtype=np.float64)
    A[np.arange(n), np.arange(n)] = s
    for v in V2:                         # A <- A H2 (right factors)
        A -= 2.0 * np.outer(A @ v, v)
    for v in V1[::-1]:                   # A <- H1 A (left factors, innermost first)
        A -= 2.0 * np.outer(v, v @ A)
    return A, V1, V2, s


def householder_apply_inverse(V1: np.ndarray, V2: np.ndarray, s: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = A^{-1} B = H2^T diag(1/s) H1^T B for the construction above."""
    X = np.array(B, dtype=np.float64, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    for v in V1:                         # H1^T = R7 ... R0 when H1 = R0 ... R7
        X -= 2.0 * np.outer(v, v @ X)
    X /= s[:, None]
    for v in V2:                         # H2^T = R7 ... R0 when H2 = R0 ... R7
        X -= 2.0 * np.outer(v, v @ X)
    return X[:, 0] if vec else X


def batch_sizes(count: int, lo: int, hi: int, seed: int, stream: int = 7) -> np.ndarray:
    """Sizes log-uniform in [lo, hi] (integers)."""
    u = uniform01(seed, stream, np.arange(count, dtype=np.uint64))
    n = np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def poisson_arrivals(rate: float, duration: float, seed: int, stream: int = 11) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    est = int(rate * duration * 1.5 + 64)
    u = uniform01(seed, stream, np.arange(est, dtype=np.uint64))
    gaps = -np.log(1.0 - u) / rate
    t = np.cumsum(gaps)
    return t[t < duration]
