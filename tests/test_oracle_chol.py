"""Pins of the oracle's Cholesky factorization and solve (A = L L^T, no
pivoting; the kernel Section 2.2 and the Conclusions name for the same
schedule) against facts fixed by mathematics, not by the oracle itself:

* exact integer factors: with L integral and its diagonal in {1, 2, 4}, every
  intermediate value of the right-looking factorization of A = L L^T is an
  integer small enough to be exact, every square root is of a perfect square
  and every division is exact, so the factor must come back bit for bit;
* numpy's Cholesky (LAPACK potrf) and solve within the backward-stable bound;
* matrices whose first non-positive pivot is known in exact arithmetic;
* the strict upper triangle is never read or written;
* special cases: n = 0, n = 1, diagonal matrices.
"""
import numpy as np
import pytest

import workloads as wl

DTYPES = [np.float64, np.float32]


def int_factor(n, seed, lo=-3, hi=3):
    """Lower-triangular integer L with diagonal entries in {1, 2, 4}."""
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(lo, hi + 1, size=(n, n)), -1).astype(np.int64)
    L[np.arange(n), np.arange(n)] = rng.choice([1, 2, 4], size=n)
    return L


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (40, 3), (129, 4)])
def test_exact_integer_factor(oracle_mod, dtype, n, seed):
    L = int_factor(n, seed)
    A = L @ L.T                                   # exact in int64
    assert np.abs(A).max() < 2 ** 22              # every partial sum exact in binary32 too
    F, info = oracle_mod.chol_factor(A.astype(np.float64), dtype=dtype)
    assert info == 0
    assert F.dtype == dtype
    np.testing.assert_array_equal(np.tril(F), L.astype(dtype))


@pytest.mark.parametrize("dtype", DTYPES)
def test_upper_triangle_untouched(oracle_mod, dtype):
    n = 50
    L = int_factor(n, 11)
    A = (L @ L.T).astype(np.float64)
    A1 = A.copy()
    A2 = A.copy()
    iu = np.triu_indices(n, 1)
    A1[iu] = 12345.5
    A2[iu] = np.nan                                # never read: no NaN may leak
    F1, i1 = oracle_mod.chol_factor(A1, dtype=dtype)
    F2, i2 = oracle_mod.chol_factor(A2, dtype=dtype)
    assert i1 == i2 == 0
    assert np.all(F1[iu] == dtype(12345.5))
    assert np.all(np.isnan(F2[iu]))
    np.testing.assert_array_equal(np.tril(F1), np.tril(F2))
    np.testing.assert_array_equal(np.tril(F1), L.astype(dtype))


@pytest.mark.parametrize("dtype", DTYPES)
def test_special_cases(oracle_mod, dtype):
    F, info = oracle_mod.chol_factor(np.zeros((0, 0)), dtype=dtype)
    assert info == 0 and F.shape == (0, 0)
    F, info = oracle_mod.chol_factor(np.array([[9.0]]), dtype=dtype)
    assert info == 0 and F[0, 0] == 3.0
    d = np.array([1.0, 2.0, 0.25, 7.0, 1e-6, 3e5])
    F, info = oracle_mod.chol_factor(np.diag(d), dtype=dtype)
    assert info == 0
    np.testing.assert_array_equal(np.diag(F), np.sqrt(d.astype(dtype)))
    np.testing.assert_array_equal(np.tril(F, -1), 0)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("j0,excess", [(0, 1), (5, 0), (17, 1), (39, 3)])
def test_info_first_nonpositive_pivot(oracle_mod, dtype, j0, excess):
    """a_{j0 j0} lowered by l_{j0 j0}^2 + excess makes the column-j0 pivot
    exactly -excess (0 when excess = 0) while every earlier pivot stays l^2."""
    n = 40
    L = int_factor(n, 21 + j0)
    A = (L @ L.T).astype(np.float64)
    A[j0, j0] -= float(L[j0, j0] ** 2 + excess)
    F, info = oracle_mod.chol_factor(A, dtype=dtype)
    assert info == j0 + 1
    np.testing.assert_array_equal(np.tril(F)[:, :j0], L[:, :j0].astype(dtype))


@pytest.mark.parametrize("dtype", DTYPES)
def test_info_nan_and_indefinite(oracle_mod, dtype):
    A = wl.matrix_spd(30, 5)
    A[12, 12] = np.nan
    _, info = oracle_mod.chol_factor(A, dtype=dtype)
    assert info == 13
    B = wl.matrix_spd(200, 6, shift=0.0)            # symmetric, indefinite
    _, info = oracle_mod.chol_factor(B, dtype=dtype)
    ev = np.linalg.eigvalsh(B)
    assert ev.min() < 0 and info >= 1
    # the leading principal minors before info are positive definite, the
    # one of order info is not (Sylvester's criterion)
    assert np.linalg.eigvalsh(B[: info - 1, : info - 1]).min() > 0 if info > 1 else True
    assert np.linalg.eigvalsh(B[:info, :info]).min() <= 1e-9 * np.abs(B).max()


@pytest.mark.parametrize("dtype,rtol", [(np.float64, 1e-12), (np.float32, 2e-5)])
@pytest.mark.parametrize("n,shift", [(64, None), (300, None), (257, 30.0)])
def test_against_lapack_potrf(oracle_mod, dtype, rtol, n, shift):
    A = wl.matrix_spd(n, 7 + n, shift=shift)
    assert np.linalg.eigvalsh(A).min() > 0
    F, info = oracle_mod.chol_factor(A, dtype=dtype)
    assert info == 0
    Lr = np.linalg.cholesky(A.astype(dtype).astype(np.float64))
    cond = np.linalg.cond(A)
    scale = np.sqrt(np.abs(np.diag(A)).max())
    err = np.abs(np.tril(F).astype(np.float64) - Lr).max() / scale
    assert err < rtol * max(1.0, cond / 10)


def test_wishart_factor_reconstructs(oracle_mod):
    """A less benign spectrum (G G^T / n + 1e-3 I): the computed factor's
    product reproduces A to the backward error bound c n eps ||A||."""
    n = 200
    G = wl.matrix_normal(n, n, 3)
    A = G @ G.T / n + 1e-3 * np.eye(n)
    F, info = oracle_mod.chol_factor(A)
    assert info == 0
    L = np.tril(F)
    assert np.abs(L @ L.T - A).max() <= 4 * n * 2.0 ** -53 * np.abs(A).max() * 10


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-14), (np.float32, 1e-6)])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (50, 1), (130, 7)])
def test_solve_against_numpy(oracle_mod, dtype, tol, n, nrhs):
    A = wl.matrix_spd(n, 40 + n)
    B = wl.matrix_uniform(n, nrhs, 41 + n)
    F, info = oracle_mod.chol_factor(A, dtype=dtype)
    assert info == 0
    X = oracle_mod.chol_solve(F, B)
    assert X.dtype == dtype
    Xr = np.linalg.solve(A.astype(dtype).astype(np.float64), B.astype(dtype).astype(np.float64))
    assert np.abs(X - Xr).max() <= tol * np.abs(Xr).max() * 10
    x = oracle_mod.chol_solve(F, B[:, 0])
    assert x.shape == (n,)


def test_solve_exact_integer(oracle_mod):
    """L with unit diagonal and integer entries: L L^T x = b has the integer
    solution it was built from, and every step is exact."""
    n = 30
    L = int_factor(n, 99, lo=-1, hi=1)
    L[np.arange(n), np.arange(n)] = 1
    x = np.random.default_rng(5).integers(-4, 5, size=(n, 3))
    A = L @ L.T
    b = A @ x
    F, info = oracle_mod.chol_factor(A.astype(np.float64))
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), L)
    X = oracle_mod.chol_solve(F, b.astype(np.float64))
    np.testing.assert_array_equal(X, x)
