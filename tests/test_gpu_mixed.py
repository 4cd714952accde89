"""GPU parity of the binary32 and low-precision factorization pieces."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import apply_piv, cuda_or_fail, lib

pytestmark = pytest.mark.gpu


def native():
    g = lib()
    from paper_2010_05975_gb300 import _native as nat
    L = nat.library()
    P, I = ctypes.c_void_p, ctypes.c_int
    L.lu_factor_f32.argtypes = [I, I, P, I, P, P, ctypes.POINTER(nat.lu_opts), P]
    L.lu_gemm_lowp.argtypes = [I, I, I, P, I, P, I, P, I, I, P, P]
    return g, nat, L


def gpu_factor_f32(A32, b, h, prec=1, defer=0):
    torch = cuda_or_fail()
    g, nat, L = native()
    dA = torch.from_numpy(A32.copy()).cuda()
    m, n = A32.shape
    piv = torch.zeros(max(min(m, n), 1), dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = nat.lu_opts(b, h, prec, defer)
    rc = L.lu_factor_f32(m, n, dA.data_ptr(), n, piv.data_ptr(), info.data_ptr(), ctypes.byref(opts),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return dA.cpu().numpy(), piv.cpu().numpy()[: min(m, n)], int(info.cpu()[0])


@pytest.mark.parametrize("n,b,h", [(64, 16, 8), (300, 32, 128), (513, 64, 64), (1000, 128, 128), (250, 100, 128),
                                   (1024, 256, 128), (2048, 256, 128), (2050, 128, 128), (1800, 90, 128)])
def test_f32_factor_bit_exact(oracle_mod, n, b, h):
    """The all-binary32 path keeps the oracle's operation order: pivots and
    factors equal the oracle's binary32 instance bit for bit.  From n ~ 1700
    the update takes the 128 x 128 binary32 tile: with 16-byte operand loads
    (n = 2048), with 4-byte loads (n = 2050: rows not 16-byte aligned) and
    with both by step (b = 90: panels alternately aligned)."""
    A = wl.matrix_uniform(n, n, seed=n, stream=32).astype(np.float32)
    LUg, pg, ig = gpu_factor_f32(A, b, h)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=h)
    np.testing.assert_array_equal(pg, po)
    assert ig == io
    np.testing.assert_array_equal(LUg, LUo)


@pytest.mark.parametrize("n,b,h", [(200, 16, 8), (600, 128, 128), (300, 100, 128)])
def test_f32_ties_and_zero_pivots(oracle_mod, n, b, h):
    """Small integers (many equal |a|, so ties fall to the smaller row
    position) and two zero columns (steps with a zero pivot update nothing)."""
    u = wl.uniform01(77, n * n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    A = (np.floor(u * 5.0) - 2.0).astype(np.float32)
    A[:, n // 3] = 0.0
    A[:, n // 3 + 5] = 0.0
    LUg, pg, ig = gpu_factor_f32(A, b, h)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=h)
    np.testing.assert_array_equal(pg, po)
    assert ig == io
    assert io > 0
    np.testing.assert_array_equal(LUg, LUo)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (129, 5), (1000, 16), (777, 40), (513, 100)])
def test_f32_solve(oracle_mod, n, nrhs):
    """Binary32 solve with binary32 factors: passes of up to 64 right-hand
    sides at padded widths 8 / 16 / 32 / 64; compared with the oracle's
    binary32 substitution within the rounding-error bound of both."""
    torch = cuda_or_fail()
    g, nat, L = native()
    A = wl.matrix_uniform(n, n, seed=n + 3, stream=40).astype(np.float32)
    B = wl.matrix_uniform(n, nrhs, seed=n + 3, stream=41).astype(np.float32)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=32, h=64)
    assert io == 0
    dLU = torch.from_numpy(LUo).cuda()
    dpiv = torch.from_numpy(po.astype(np.int32)).cuda()
    dB = torch.from_numpy(B.copy()).cuda()
    from paper_2010_05975_gb300 import api
    api.lu_solve_f32(dLU, dpiv, dB)
    torch.cuda.synchronize()
    X = dB.cpu().numpy().astype(np.float64)
    Xo = oracle_mod.lu_solve_f32(LUo, po, B).astype(np.float64)
    cond = np.linalg.cond(A.astype(np.float64))
    eps32 = np.finfo(np.float32).eps
    assert np.abs(X - Xo).max() <= 64 * n * eps32 * cond * np.abs(Xo).max()
    assert oracle_mod.backward_error(A.astype(np.float64), B.astype(np.float64), X).max() <= 20 * n * eps32


def run_gemm_lowp(L32, U32, C32, fp8):
    torch = cuda_or_fail()
    g, nat, Lb = native()
    M, K = L32.shape
    N = U32.shape[1]
    dL = torch.from_numpy(L32.copy()).cuda()
    dU = torch.from_numpy(U32.copy()).cuda()
    dC = torch.from_numpy(C32.copy()).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = Lb.lu_gemm_lowp(M, N, K, dL.data_ptr(), K, dU.data_ptr(), N, dC.data_ptr(), N,
                         3 if fp8 else 2, st.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("fp8", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 128, 256), (300, 200, 256), (129, 513, 64), (1000, 1000, 256),
                                   (77, 140, 16), (4096, 700, 200)])
def test_gemm_lowp_matches_oracle(oracle_mod, fp8, M, N, K):
    """tcgen05 update vs the binary64-summed reference of the same quantized
    operands.  Tolerance: fp32 accumulation of K products and one rounding of
    C, |d| <= 2^-22 |Cref| + (K + 2) 2^-21 * s sum|qL qU|."""
    rng = np.random.default_rng(M * 7 + N + K)
    L = rng.standard_normal((M, K)).astype(np.float32)
    U = (rng.standard_normal((K, N)) * 30).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    Cg = run_gemm_lowp(L, U, C, fp8)
    Cref, Sabs = oracle_mod.gemm_lowp(L, U, C, fp8=fp8)
    tol = 2.0 ** -22 * np.abs(Cref) + (K + 2) * 2.0 ** -21 * Sabs + 1e-30
    err = np.abs(Cg.astype(np.float64) - Cref)
    assert (err <= tol).all(), (err / tol).max()


def _residual(A, LU, piv):
    n = A.shape[0]
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    return np.linalg.norm(apply_piv(A.astype(np.float64), piv) - L @ U) / np.linalg.norm(A)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n,b", [(512, 128), (1000, 256), (2048, 256)])
def test_lowp_factor_against_oracle(oracle_mod, prec, n, b):
    """bf16 / fp8 Schur updates.  Step 0 sees identical binary32 inputs on
    both sides, so its b pivots agree exactly; later steps start from values
    that differ by fp32 accumulation order, which moves some bf16/fp8
    roundings, so the factors are compared through their backward error:
    within a factor 2 of the oracle's own mixed-precision factorization."""
    A = wl.matrix_uniform(n, n, seed=n + prec).astype(np.float32)
    LUg, pg, ig = gpu_factor_f32(A, b, 128, prec=prec)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=128, lowp=prec - 1)
    assert ig == io == 0
    assert np.isfinite(LUg).all()
    assert ((pg >= np.arange(n)) & (pg < n)).all()
    np.testing.assert_array_equal(pg[:b], po[:b])
    rg, ro = _residual(A, LUg, pg), _residual(A, LUo, po)
    assert 0.5 * ro <= rg <= 2.0 * ro, (rg, ro)


# --- closed forms: the mixed-precision factorization bit for bit ------------

from tests import lowp_closed_form as cf  # noqa: E402


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n,b,h", [(1100, 128, 128), (1100, 256, 128), (777, 128, 64)])
def test_lowp_factor_exact_closed_form_bitwise(oracle_mod, prec, n, b, h):
    """Operands exact in bf16 / e4m3 and partial sums exact in binary32:
    whatever order the tensor cores add in, the GPU returns P = I and the
    closed-form L and U bit for bit, as the oracle does."""
    A, LU = cf.exact_factors(n)
    LUg, pg, ig = gpu_factor_f32(A, b, h, prec=prec)
    assert ig == 0
    np.testing.assert_array_equal(pg, np.arange(n))
    np.testing.assert_array_equal(LUg, LU)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=h, lowp=prec - 1)
    np.testing.assert_array_equal(LUg, LUo)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("b", [128, 256])
def test_lowp_factor_rounded_first_update_bitwise(oracle_mod, prec, b):
    """The first tensor-core update rounds L21 and U12 (bf16, or e4m3 with the
    step's tile scales, some values on the subnormal grid); its result is
    exact in binary32, so the trailing block must come out as the diagonal D
    and the factors as the closed form, bit for bit."""
    n = b + 600
    A, LU = cf.rounded_first_update(n, b, prec == 3)
    LUg, pg, ig = gpu_factor_f32(A, b, 128, prec=prec)
    assert ig == 0
    np.testing.assert_array_equal(pg, np.arange(n))
    np.testing.assert_array_equal(LUg, LU)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=128, lowp=prec - 1)
    np.testing.assert_array_equal(LUg, LUo)


# --- deferred trailing updates: the same factors for every deferral ---------

@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n,b", [(1100, 128), (2048, 128), (1500, 256), (777, 128)])
def test_lowp_deferred_updates_bitwise(prec, n, b):
    """Holding back up to 4 panels' updates and applying them in one pass
    (each panel into its own accumulator, applied in step order) must give
    the per-step factors bit for bit, on generic inputs where every rounding
    counts.  n = 777 has rows that are not 16-byte aligned (the epilogue's
    per-thread path); the others use the TMA epilogue."""
    A = wl.matrix_uniform(n, n, seed=n + 11 * prec, stream=50).astype(np.float32)
    ref, pref, iref = gpu_factor_f32(A, b, 128, prec=prec, defer=1)
    assert iref == 0
    for d in (2, 3, 4):
        LUg, pg, ig = gpu_factor_f32(A, b, 128, prec=prec, defer=d)
        assert ig == 0
        np.testing.assert_array_equal(pg, pref)
        np.testing.assert_array_equal(LUg, ref)


@pytest.mark.parametrize("prec", [2, 3])
def test_lowp_closed_form_every_deferral(oracle_mod, prec):
    """The exact closed form comes back bit for bit at every deferral."""
    A, LU = cf.exact_factors(1100)
    for d in (1, 2, 3, 4):
        LUg, pg, ig = gpu_factor_f32(A, 128, 128, prec=prec, defer=d)
        assert ig == 0
        np.testing.assert_array_equal(pg, np.arange(1100))
        np.testing.assert_array_equal(LUg, LU)
