"""Mixed-precision factorization + binary64 refinement (through the C ABI).

Matrices A = H1 diag(s) H2 (8 seeded Householder reflectors per side,
s_i = kappa^(-i/(n-1))), so kappa_2(A) = kappa and A^{-1} is known in closed
form.  The bar: max backward error <= 1e-12 (recomputed by the oracle), and
the forward error against the closed-form solution within 10 * kappa * 1e-12.
"""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu

BF16, FP8, F32 = 2, 3, 1


def make_problem(n, kappa, nrhs, seed):
    A, V1, V2, s = wl.householder_diag(n, kappa, seed=seed)
    Xt = wl.matrix_normal(n, nrhs, seed=seed + 1000)
    B = A @ Xt
    return A, B, Xt


@pytest.mark.parametrize("prec", [BF16, FP8, F32])
@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e8])
def test_ir_reaches_1e12(oracle_mod, prec, kappa):
    torch = cuda_or_fail()
    g = lib()
    n, nrhs = 1024, 16
    A, B, Xt = make_problem(n, kappa, nrhs, seed=int(np.log10(kappa)))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    X, res = g.ir_solve(dA, dB, precision=prec)
    Xg = X.cpu().numpy()
    eta = oracle_mod.backward_error(A, B, Xg)
    assert res["path"] in (0, 1), res
    assert res["eta"] <= 1e-12 and eta.max() <= 1e-12, (res, eta.max())
    fwd = np.abs(Xg - Xt).max(axis=0) / np.abs(Xt).max(axis=0)
    assert fwd.max() <= 10 * kappa * 1e-12, (fwd.max(), res)


def test_ir_matches_oracle_solution(oracle_mod):
    """Same X as the oracle's binary64 LU solve, to the conditioning bound."""
    torch = cuda_or_fail()
    g = lib()
    n, nrhs, kappa = 512, 4, 1e4
    A, B, Xt = make_problem(n, kappa, nrhs, seed=77)
    X, res = g.ir_solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), precision=BF16)
    LU, piv, _ = oracle_mod.lu_factor(A, b=32, h=128)
    Xo = oracle_mod.lu_solve(LU, piv, B)
    d = np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max()
    assert d <= 10 * kappa * 2e-12, d


@pytest.mark.parametrize("n,nrhs", [(1, 1), (100, 3), (777, 9), (2048, 16)])
def test_residual_kernel(oracle_mod, n, nrhs):
    """lu_residual: R = B - A X and eta against the oracle's definition."""
    torch = cuda_or_fail()
    g = lib()
    A = wl.matrix_uniform(n, n, seed=n)
    X = wl.matrix_normal(n, nrhs, seed=n + 1)
    B = wl.matrix_normal(n, nrhs, seed=n + 2)
    R, eta = g.lu_residual(torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda())
    torch.cuda.synchronize()
    Rr = B - A @ X
    scale = np.abs(A).sum(axis=1).max() * np.abs(X).max()
    assert np.abs(R.cpu().numpy() - Rr).max() <= 4 * n * 2.0 ** -53 * scale
    eo = oracle_mod.backward_error(A, B, X)
    np.testing.assert_allclose(eta.cpu().numpy(), eo, rtol=1e-12)


@pytest.mark.parametrize("prec,kappa", [(FP8, 1e2), (BF16, 1e4), (BF16, 1e6)])
@pytest.mark.parametrize("products", [0, 1, 2])
def test_ir_krylov_products(oracle_mod, prec, kappa, products):
    """Every choice of Krylov products reaches 1e-12: binary32 multiplies
    (2), binary64 (1), or the adaptive rule (0), which runs its first FGMRES
    cycle with binary32 multiplies and stays with them while they pay."""
    torch = cuda_or_fail()
    g = lib()
    n, nrhs = 1024, 8
    A, B, Xt = make_problem(n, kappa, nrhs, seed=40 + int(np.log10(kappa)))
    X, res = g.ir_solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), precision=prec,
                        krylov_products=products)
    eta = oracle_mod.backward_error(A, B, X.cpu().numpy())
    assert res["eta"] <= 1e-12 and eta.max() <= 1e-12, (res, eta.max())
    if res["path"] == 1:
        if products == 1:
            assert res["cycles32"] == 0 and res["cycles64"] >= 1, res
        else:
            assert res["cycles32"] >= 1, res
        if products == 2:
            assert res["cycles64"] == 0, res


def test_ir_rejects_bad_krylov_option():
    torch = cuda_or_fail()
    g = lib()
    from paper_2010_05975_gb300 import _native as nat
    A = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.LuError):
        g.ir_solve(A, torch.ones(8, 1, dtype=torch.float64, device="cuda"), krylov_products=3)


@pytest.mark.parametrize("inner", [-1, 0, 5])
def test_ir_inner_steps(oracle_mod, inner):
    """Classical steps with and without the binary32-product inner steps all
    reach 1e-12; with them (bf16, kappa = 1e2) fewer binary64 residuals are
    needed than without."""
    torch = cuda_or_fail()
    g = lib()
    n, nrhs = 1024, 8
    A, B, Xt = make_problem(n, 1e2, nrhs, seed=61)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    X, res = g.ir_solve(dA, dB, precision=BF16, inner_steps=inner)
    eta = oracle_mod.backward_error(A, B, X.cpu().numpy())
    assert res["eta"] <= 1e-12 and eta.max() <= 1e-12, (res, eta.max())
    if inner < 0:
        assert res["inner_steps"] == 0
    else:
        _, plain = g.ir_solve(dA, dB, precision=BF16, inner_steps=-1)
        if res["path"] == 0 and plain["path"] == 0:
            assert res["inner_steps"] >= 1 and res["iters"] < plain["iters"], (res, plain)
