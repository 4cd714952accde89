"""Parity of the Cholesky factorization (C ABI chol_factor / chol_factor_f32)
with the CPU oracle: the lower triangle bit for bit in binary64 and binary32
(the kernels keep the oracle's per-element order: update terms in ascending
column, then the square root or one division), info equal, and the strict
upper triangle of the device buffer untouched (filled with NaN, which must
neither be read into L nor be overwritten)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu


def run_gpu(A, b=0, lda=None, dtype=np.float64):
    torch = cuda_or_fail()
    g = lib()
    n = A.shape[0]
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    ld = n if lda is None else lda
    buf = torch.full((n, max(ld, 1)), float("nan"), dtype=tdt, device="cuda")
    Ah = np.tril(A.astype(dtype)) + np.triu(np.full_like(A, np.nan, dtype=dtype), 1)
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(Ah)).cuda()
    dA = buf[:, :n]
    info = g.chol_factor(dA, b=b)
    torch.cuda.synchronize()
    out = buf.cpu().numpy()
    if ld > n:
        assert np.isnan(out[:, n:]).all(), "padding columns were written"
    return out[:, :n], int(info.cpu()[0])


def check(oracle_mod, A, b, lda=None, dtype=np.float64):
    Fg, ig = run_gpu(A, b, lda, dtype)
    Fo, io = oracle_mod.chol_factor(A, dtype=dtype)
    assert ig == io
    n = A.shape[0]
    iu = np.triu_indices(n, 1)
    assert np.isnan(Fg[iu]).all(), "strict upper triangle was written"
    cols = n if io == 0 else io - 1
    Lg = np.tril(Fg)[:, :cols]
    Lo = np.tril(Fo)[:, :cols]
    np.testing.assert_array_equal(Lg, Lo)
    return Fg, ig


@pytest.mark.parametrize("n,b,lda", [(1, 0, None), (5, 0, None), (64, 64, None), (130, 32, None), (300, 7, None),
                                     (515, 64, 520), (1000, 128, None), (1023, 128, 1030), (2000, 0, None),
                                     (777, 100, None)])
def test_f64_bit_exact(oracle_mod, n, b, lda):
    A = wl.matrix_spd(n, seed=n)
    check(oracle_mod, A, b, lda)


@pytest.mark.parametrize("n,b,lda", [(1, 0, None), (200, 64, None), (515, 128, None), (1000, 96, None),
                                     (1536, 128, None), (3000, 128, None), (2500, 100, 2503), (2200, 90, None)])
def test_f32_bit_exact(oracle_mod, n, b, lda):
    """From n ~ 1800 the symmetric update takes the 128 x 128 binary32 tile:
    16-byte operand loads (n = 3000), 4-byte loads (lda = 2503) and both by
    step (b = 90)."""
    A = wl.matrix_spd(n, seed=n + 1)
    check(oracle_mod, A, b, lda, dtype=np.float32)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_exact_integer_factor(oracle_mod, dtype):
    """A = L L^T with integral L (diagonal in {1, 2, 4}) comes back as L."""
    n = 300
    rng = np.random.default_rng(8)
    L = np.tril(rng.integers(-2, 3, size=(n, n)), -1).astype(np.int64)
    L[np.arange(n), np.arange(n)] = rng.choice([1, 2, 4], size=n)
    A = (L @ L.T).astype(np.float64)
    assert np.abs(A).max() < 2 ** 22
    Fg, ig = check(oracle_mod, A, 64, dtype=dtype)
    assert ig == 0
    np.testing.assert_array_equal(np.tril(Fg), L.astype(dtype))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n,b,shift", [(400, 64, 0.0), (1000, 128, 5.0), (129, 32, 1.0)])
def test_indefinite_info(oracle_mod, dtype, n, b, shift):
    """Symmetric indefinite inputs: the same first non-positive pivot and the
    same columns before it."""
    A = wl.matrix_spd(n, seed=3 * n, shift=shift)
    _, ig = check(oracle_mod, A, b, dtype=dtype)
    assert ig >= 1


@pytest.mark.parametrize("j0", [0, 63, 64, 200])
def test_zero_and_negative_pivot_positions(oracle_mod, j0):
    """An exactly zero pivot at a block boundary, inside a block, and a NaN."""
    n = 260
    rng = np.random.default_rng(j0)
    L = np.tril(rng.integers(-2, 3, size=(n, n)), -1).astype(np.int64)
    L[np.arange(n), np.arange(n)] = rng.choice([1, 2, 4], size=n)
    A = (L @ L.T).astype(np.float64)
    A[j0, j0] -= float(L[j0, j0] ** 2)          # pivot j0 becomes exactly 0
    _, ig = check(oracle_mod, A, 64)
    assert ig == j0 + 1
    A2 = (L @ L.T).astype(np.float64)
    A2[j0, j0] = np.nan
    _, ig2 = check(oracle_mod, A2, 64)
    assert ig2 == j0 + 1


def test_independent_of_panel_width():
    """Bit-identical factors for b = 128, 64, 33 at n = 4096 (the per-element
    order does not depend on the blocking)."""
    n = 4096
    A = wl.matrix_spd(n, seed=77)
    ref, _ = run_gpu(A, 128)
    for b in (64, 33):
        Fb, ib = run_gpu(A, b)
        assert ib == 0
        np.testing.assert_array_equal(np.tril(Fb), np.tril(ref))


def test_empty_and_stream():
    torch = cuda_or_fail()
    g = lib()
    A = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    info = g.chol_factor(A)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    s = torch.cuda.Stream()
    n = 300
    Ah = wl.matrix_spd(n, seed=4)
    dA = torch.from_numpy(Ah).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        info = g.chol_factor(dA, stream=s)
    s.synchronize()
    Lg = torch.tril(dA).cpu().numpy()
    assert int(info.cpu()[0]) == 0
    assert np.abs(Lg @ Lg.T - Ah).max() <= 8 * n * 2.0 ** -53 * np.abs(Ah).max()


EPS = 2.0 ** -53


@pytest.mark.parametrize("dtype,eps", [(np.float64, EPS), (np.float32, 2.0 ** -24)])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (100, 1), (257, 5), (1030, 16), (700, 40), (300, 100), (2000, 3)])
def test_solve_against_oracle(oracle_mod, dtype, eps, n, nrhs):
    """chol_solve with the oracle's factor: the solution within the forward
    error bound of the oracle's substitution, and a backward error of a
    backward-stable solve.  (The GPU applies inverted diagonal blocks, so the
    rounding differs from plain substitution.)"""
    torch = cuda_or_fail()
    g = lib()
    A = wl.matrix_spd(n, seed=n, stream=1, shift=n / 4 + 3 * np.sqrt(n) + 1)
    B = wl.matrix_uniform(n, nrhs, seed=n, stream=2)
    Fo, io = oracle_mod.chol_factor(A, dtype=dtype)
    assert io == 0
    Xo = oracle_mod.chol_solve(Fo, B)
    Fd = np.tril(Fo) + np.triu(np.full_like(Fo, np.nan), 1)      # upper never read
    dL = torch.from_numpy(np.ascontiguousarray(Fd)).cuda()
    dB = torch.from_numpy(B.astype(dtype)).cuda()
    g.chol_solve(dL, dB)
    torch.cuda.synchronize()
    X = dB.cpu().numpy().astype(np.float64)
    assert np.isfinite(X).all()
    cond = np.linalg.cond(A)
    assert np.abs(X - Xo).max() <= 64 * n * eps * cond * np.abs(Xo).max()
    Ad = A.astype(dtype).astype(np.float64)
    R = B.astype(dtype).astype(np.float64) - Ad @ X
    eta = np.abs(R).max(axis=0) / (np.abs(Ad).sum(axis=1).max() * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))
    assert eta.max() <= 20 * n * eps


def test_solve_vector_after_gpu_factor(oracle_mod):
    """The public pair chol_factor -> chol_solve on a 1-D right-hand side:
    the factor is the oracle's bit for bit, the solution within the forward
    error bound of the oracle's."""
    torch = cuda_or_fail()
    g = lib()
    n = 777
    A = wl.matrix_spd(n, seed=5, shift=100.0)
    b = wl.matrix_uniform(n, 1, seed=6)[:, 0]
    dA = torch.from_numpy(A.copy()).cuda()
    info = g.chol_factor(dA)
    db = torch.from_numpy(b.copy()).cuda()
    g.chol_solve(dA, db)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    Fo, _ = oracle_mod.chol_factor(A)
    np.testing.assert_array_equal(torch.tril(dA).cpu().numpy(), np.tril(Fo))
    xo = oracle_mod.chol_solve(Fo, b)
    x = db.cpu().numpy()
    assert x.shape == (n,)
    assert np.abs(x - xo).max() <= 64 * n * EPS * np.linalg.cond(A) * np.abs(xo).max()


# --- full size: the benchmark's configuration (n = 32768, b = 128) -----------

N_FULL, B_FULL, K_FULL = 32768, 128, 2048


@pytest.fixture(scope="module")
def chol_full():
    torch = cuda_or_fail()
    g = lib()
    A = wl.matrix_spd(N_FULL, seed=3)
    dA = torch.from_numpy(A).cuda()
    info = g.chol_factor(dA, b=B_FULL)
    torch.cuda.synchronize()
    return A, dA, int(info.cpu()[0])


def test_full_size_sampled_rows_match_oracle(oracle_mod, chol_full):
    """Columns < K of row i of L depend only on A[:K, :K] and A[i, :K] (and
    a_ii for i < K), so the oracle's factor of the principal submatrix on
    {0..K-1} and 48 sampled rows gives those rows' leading K columns, with
    the same per-element operation order: compare them bit for bit."""
    A, dA, info = chol_full
    assert info == 0
    rng = np.random.default_rng(12)
    rows = np.unique(np.concatenate([[K_FULL, N_FULL - 1],
                                     rng.choice(np.arange(K_FULL + 1, N_FULL - 1), 46, replace=False)]))
    sel = np.concatenate([np.arange(K_FULL), rows])
    oracle_mod.set_threads(0)
    Fo, io = oracle_mod.chol_factor(np.ascontiguousarray(A[np.ix_(sel, sel)]))
    assert io == 0
    L11 = np.tril(dA[:K_FULL, :K_FULL].cpu().numpy())
    np.testing.assert_array_equal(L11, np.tril(Fo[:K_FULL, :K_FULL]))
    import torch
    Lr = dA[torch.from_numpy(rows).cuda(), :K_FULL].cpu().numpy()
    np.testing.assert_array_equal(Lr, Fo[K_FULL:, :K_FULL])


def test_full_size_probe(chol_full):
    """||A x - L (L^T x)|| / (||A|| ||x||) <= 20 n 2^-53 for 8 Gaussian x."""
    import torch
    A, dA, info = chol_full
    dA0 = torch.from_numpy(A).cuda()
    L = torch.tril(dA)
    X = torch.randn(N_FULL, 8, dtype=torch.float64, device="cuda",
                    generator=torch.Generator("cuda").manual_seed(6))
    r = torch.linalg.norm(dA0 @ X - L @ (L.T @ X)) / (torch.linalg.norm(dA0) * torch.linalg.norm(X))
    assert float(r) <= 20 * N_FULL * 2.0 ** -53, float(r)


def test_full_size_solve(chol_full):
    """16 right-hand sides at n = 32768: normwise backward error of the solve."""
    import torch
    g = lib()
    A, dA, info = chol_full
    dA0 = torch.from_numpy(A).cuda()
    B = torch.from_numpy(wl.matrix_uniform(N_FULL, 16, seed=9)).cuda()
    X = B.clone()
    g.chol_solve(dA, X)
    torch.cuda.synchronize()
    R = B - dA0 @ X
    eta = R.abs().amax(0) / (dA0.abs().sum(1).amax() * X.abs().amax(0) + B.abs().amax(0))
    assert float(eta.max()) <= 20 * N_FULL * 2.0 ** -53, float(eta.max())
