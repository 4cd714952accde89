"""Parity of the binary64 CUDA path (through the C ABI) with the CPU oracle.

The bar: pivots bit-exact; factor entries within 1e-10 of the oracle
(relative to the entry or its row's largest entry);
||PA - LU||_F / ||A||_F <= 20 n 2^-53.  The kernels keep the oracle's
per-element operation order, so bit-identical factors are also checked.
"""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import apply_piv, cuda_or_fail, factor_close, lib, split_lu, to_dev

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def run_gpu(A, b, h, lda=None):
    torch = cuda_or_fail()
    g = lib()
    dA, _ = to_dev(A, lda)
    piv, info = g.lu_factor_ex(dA, b=b, h=h)
    torch.cuda.synchronize()
    return dA.cpu().numpy(), piv.cpu().numpy(), int(info.cpu()[0])


def check_against_oracle(oracle_mod, A, b, h, lda=None, exact=True):
    LUg, pg, ig = run_gpu(A, b, h, lda)
    LUo, po, io = oracle_mod.lu_factor(A, b=b, h=h)
    np.testing.assert_array_equal(pg, po)
    assert ig == io
    ok, nbad = factor_close(LUg, LUo)
    assert ok, f"{nbad} entries outside 1e-10"
    m, n = A.shape
    L, U = split_lu(LUg)
    res = np.linalg.norm(apply_piv(A, pg) - L @ U) / np.linalg.norm(A)
    assert res <= 20 * max(m, n) * EPS
    if exact:
        np.testing.assert_array_equal(LUg, LUo)
    return LUg, pg


def test_c1_factor_and_solve(oracle_mod):
    """N = 512, b = 32, h = 128, Uniform[-1,1] seed 0, b = A ones(N)."""
    torch = cuda_or_fail()
    g = lib()
    n = 512
    A = wl.matrix_uniform(n, n, seed=0)
    LUg, pg = check_against_oracle(oracle_mod, A, 32, 128)
    rhs = A @ np.ones(n)
    dLU = torch.from_numpy(LUg).cuda()
    dpiv = torch.from_numpy(pg.astype(np.int32)).cuda()
    dB = torch.from_numpy(rhs.copy()).cuda()
    g.lu_solve(dLU, dpiv, dB)
    torch.cuda.synchronize()
    x = dB.cpu().numpy()
    LUo, po, _ = oracle_mod.lu_factor(A, b=32, h=128)
    xo = oracle_mod.lu_solve(LUo, po, rhs)
    assert np.abs(x - xo).max() <= 1e-12 * np.abs(xo).max() * 100
    assert np.abs(x - 1.0).max() <= 1e-10
    eta = oracle_mod.backward_error(A, rhs, x)
    assert eta.max() <= 20 * n * EPS


@pytest.mark.parametrize("n,b,h", [(1, 1, 1), (2, 1, 1), (17, 4, 3), (33, 8, 8), (100, 32, 128), (129, 16, 4),
                                   (257, 32, 128), (300, 64, 16), (513, 256, 128), (640, 128, 200), (700, 256, 64)])
def test_square_ragged(oracle_mod, n, b, h):
    A = wl.matrix_normal(n, n, seed=n + b, stream=h)
    check_against_oracle(oracle_mod, A, b, h)


@pytest.mark.parametrize("m,n,b,h", [(300, 120, 32, 16), (120, 300, 32, 16), (1000, 256, 64, 128), (77, 500, 16, 8)])
def test_rectangular(oracle_mod, m, n, b, h):
    A = wl.matrix_uniform(m, n, seed=m, stream=n)
    check_against_oracle(oracle_mod, A, b, h)


def test_padded_leading_dimension(oracle_mod):
    n = 200
    A = wl.matrix_uniform(n, n, seed=5)
    check_against_oracle(oracle_mod, A, 32, 32, lda=n + 13)


def test_zero_column_info(oracle_mod):
    n = 96
    A = wl.matrix_uniform(n, n, seed=6)
    A[:, 40] = 0.0
    LUg, pg, ig = run_gpu(A, 32, 16)
    LUo, po, io = oracle_mod.lu_factor(A, b=32, h=16)
    assert ig == io == 41
    np.testing.assert_array_equal(pg, po)
    assert np.isfinite(LUg).all()
    np.testing.assert_array_equal(LUg, LUo)


@pytest.mark.parametrize("n,b,h", [(700, 256, 128), (300, 64, 16)])
def test_cluster_nodes_ties_and_zero_pivots(oracle_mod, n, b, h):
    """Tournament nodes spread over a cluster: small integers (many equal
    |a|; ties go to the smaller row position) and two zero columns (steps
    with a zero pivot update nothing) give the oracle's factors exactly."""
    u = wl.uniform01(91, n * n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    A = np.floor(u * 5.0) - 2.0
    A[:, n // 3] = 0.0
    A[:, n // 3 + 5] = 0.0
    LUg, pg, ig = run_gpu(A, b, h)
    LUo, po, io = oracle_mod.lu_factor(A, b=b, h=h)
    np.testing.assert_array_equal(pg, po)
    assert ig == io
    assert io > 0
    np.testing.assert_array_equal(LUg, LUo)


def test_permutation_matrix_exact():
    n = 160
    perm = np.argsort(wl.uniform01(9, n, np.arange(n, dtype=np.uint64)))
    Q = np.zeros((n, n))
    Q[np.arange(n), perm] = 1.0
    LUg, pg, ig = run_gpu(Q, 32, 8)
    assert ig == 0
    np.testing.assert_array_equal(LUg, np.eye(n))
    np.testing.assert_array_equal(apply_piv(Q, pg), np.eye(n))


def test_closed_form_identity_pivots():
    """A = L U with |l| <= 1/2, |u_jj| >= 1 and dyadic entries: P = I and the
    factors come back exactly (a closed form, not the oracle)."""
    n = 384
    ul = wl.uniform01(5, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    uu = wl.uniform01(6, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    L = np.tril(np.floor(ul * 17 - 8.5 + 0.5) / 16.0, -1) + np.eye(n)
    U = np.triu(np.floor(uu * 33 - 16.5 + 0.5) / 16.0, 1)
    d = np.floor(np.diag(uu) * 17) / 16.0 + 1.0
    U += np.diag(np.where(np.arange(n) % 2 == 0, d, -d))
    LUg, pg, ig = run_gpu(L @ U, 64, 16)
    np.testing.assert_array_equal(pg, np.arange(n))
    Lg, Ug = split_lu(LUg)
    np.testing.assert_array_equal(Lg, L)
    np.testing.assert_array_equal(Ug, U)


def test_deterministic_repeats():
    n = 600
    A = wl.matrix_normal(n, n, seed=3)
    outs = [run_gpu(A, 64, 32) for _ in range(4)]
    for LU, p, _ in outs[1:]:
        np.testing.assert_array_equal(p, outs[0][1])
        np.testing.assert_array_equal(LU, outs[0][0])


def test_empty_matrix():
    torch = cuda_or_fail()
    g = lib()
    A = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    piv, info = g.lu_factor(A)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0


@pytest.mark.parametrize("n,nrhs", [(1, 1), (64, 1), (65, 3), (500, 8), (1030, 64), (300, 33), (257, 65),
                                    (1030, 130), (200, 384)])
def test_solve_multi_rhs(oracle_mod, n, nrhs):
    torch = cuda_or_fail()
    g = lib()
    A = wl.matrix_uniform(n, n, seed=n, stream=1)
    B = wl.matrix_uniform(n, nrhs, seed=n, stream=2)
    LUo, po, _ = oracle_mod.lu_factor(A, b=32, h=64)
    dLU = torch.from_numpy(LUo).cuda()
    dpiv = torch.from_numpy(po.astype(np.int32)).cuda()
    dB = torch.from_numpy(B.copy()).cuda()
    g.lu_solve(dLU, dpiv, dB)
    torch.cuda.synchronize()
    X = dB.cpu().numpy()
    Xo = oracle_mod.lu_solve(LUo, po, B)
    cond = np.linalg.cond(A)
    assert np.abs(X - Xo).max() <= 64 * n * EPS * cond * np.abs(Xo).max()
    assert oracle_mod.backward_error(A, B, X).max() <= 20 * n * EPS
