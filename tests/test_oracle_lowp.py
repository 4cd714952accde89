"""Pins of the oracle's binary32 factorization and low-precision pieces."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import workloads as wl


def test_round_bf16_matches_torch(oracle_mod):
    """bfloat16 rounding (nearest, ties even) equals torch's conversion."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([1.0, 1.00390625, 1.0078125, 1.01171875, -1.01171875, 3.0e38], np.float32)])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle_mod.round_lowp(x, fp8=False), ref)


def test_round_e4m3_matches_torch_in_range(oracle_mod):
    """e4m3 rounding equals torch's float8_e4m3fn conversion for |x| <= 448."""
    rng = np.random.default_rng(1)
    x = (rng.uniform(-448, 448, 20000) * 2.0 ** rng.integers(-14, 1, 20000)).astype(np.float32)
    x = np.concatenate([x, np.array([0.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11, 448.0, -448.0, 1.0625, 1.1875],
                                    np.float32)])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle_mod.round_lowp(x, fp8=True), ref)


def test_round_e4m3_hand_cases(oracle_mod):
    """Ties to even on the 1/8 grid, saturation above 448."""
    x = np.array([1.0625, 1.1875, 464.0, 470.0, 1e6, -1e6, 2.0 ** -10], np.float32)
    # 1.0625 = 1 + 1/16 (tie) -> 1.0 ; 1.1875 = 1.125 + 1/16 (tie) -> 1.25 ; big -> 448 ; 2^-10 (tie) -> 0
    np.testing.assert_array_equal(oracle_mod.round_lowp(x, fp8=True),
                                  np.array([1.0, 1.25, 448.0, 448.0, 448.0, -448.0, 0.0], np.float32))


def test_e4m3_exponent(oracle_mod):
    """Smallest e with maxabs * 2^-e <= 448."""
    assert oracle_mod.e4m3_exponent(448.0) == 0
    assert oracle_mod.e4m3_exponent(449.0) == 1
    assert oracle_mod.e4m3_exponent(224.0) == -1
    assert oracle_mod.e4m3_exponent(225.0) == 0
    assert oracle_mod.e4m3_exponent(1.0) == -8
    assert oracle_mod.e4m3_exponent(0.0) == 0


@pytest.mark.parametrize("fp8", [False, True])
def test_gemm_lowp_exact_operands(oracle_mod, fp8):
    """Operands exactly representable after scaling: the update equals the
    binary64 product C - L U."""
    rng = np.random.default_rng(2)
    M, N, K = 300, 270, 64
    L = (rng.integers(-7, 8, (M, K)) * 0.25).astype(np.float32)     # <= 4 significant bits
    U = (rng.integers(-7, 8, (K, N)) * 0.5).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    Cref, Sabs = oracle_mod.gemm_lowp(L, U, C, fp8=fp8)
    np.testing.assert_array_equal(Cref, C.astype(np.float64) - L.astype(np.float64) @ U.astype(np.float64))
    np.testing.assert_array_equal(Sabs, np.abs(L.astype(np.float64)) @ np.abs(U.astype(np.float64)))


def test_gemm_lowp_scale_blocks(oracle_mod):
    """fp8: one power-of-two scale per 256-row block of L and 256-column block
    of U; a block of huge values does not change its neighbours' rounding."""
    M, N, K = 512, 300, 8
    L = np.full((M, K), 1.0, np.float32)
    L[256:] = 1000.0                                    # second block scaled by 2^2
    U = np.full((K, N), 0.5, np.float32)
    C = np.zeros((M, N), np.float32)
    Cref, _ = oracle_mod.gemm_lowp(L, U, C, fp8=True)
    np.testing.assert_array_equal(Cref[:256], -4.0)     # 8 * 1 * 0.5
    # 1000 / 4 = 250 -> e4m3 grid spacing 16 -> 256 -> 1024 after scaling
    np.testing.assert_array_equal(Cref[256:], -8 * 1024.0 * 0.5)


@pytest.mark.parametrize("n,h", [(64, 8), (150, 128)])
def test_f32_b1_equals_sgetrf(oracle_mod, n, h):
    A = wl.matrix_uniform(n, n, seed=40 + n).astype(np.float32)
    LU, piv, info = oracle_mod.lu_factor_f32(A, b=1, h=h)
    lu_ref, ipiv = sla.lu_factor(A)
    assert lu_ref.dtype == np.float32
    np.testing.assert_array_equal(piv, ipiv)
    np.testing.assert_allclose(LU, lu_ref, rtol=0, atol=2e-5 * np.abs(lu_ref).max())


def test_f32_closed_form_exact(oracle_mod):
    n = 96
    ul = wl.uniform01(15, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    uu = wl.uniform01(16, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    L = np.tril(np.floor(ul * 17 - 8.5 + 0.5) / 16.0, -1) + np.eye(n)
    U = np.triu(np.floor(uu * 33 - 16.5 + 0.5) / 16.0, 1) + np.diag(np.floor(np.diag(uu) * 17) / 16.0 + 1.0)
    A = (L @ U).astype(np.float32)
    assert np.array_equal(A.astype(np.float64), L @ U)
    LU, piv, info = oracle_mod.lu_factor_f32(A, b=16, h=8)
    np.testing.assert_array_equal(piv, np.arange(n))
    np.testing.assert_array_equal(np.tril(LU, -1) + np.eye(n), L.astype(np.float32))
    np.testing.assert_array_equal(np.triu(LU), U.astype(np.float32))


# --- the mixed-precision factorization (Section 7.2 FactorizeA11 with the
# low-precision operands of the mixed-precision reading), pinned by closed
# forms whose factors are known before the factorization runs --------------

from tests import lowp_closed_form as cf  # noqa: E402


@pytest.mark.parametrize("lowp", [1, 2])
@pytest.mark.parametrize("n,b,h", [(1100, 128, 128), (1100, 256, 128), (777, 128, 64)])
def test_lowp_factor_exact_closed_form(oracle_mod, lowp, n, b, h):
    """A = L U whose operands are exact in bf16 and e4m3 and whose partial
    sums are exact in binary32: every step is exact, so P = I and the factors
    are L and U bit for bit.  Row / column classes 4x apart make a value that
    takes another tile's fp8 scale saturate, so a misplaced scale fails."""
    A, LU = cf.exact_factors(n)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=h, lowp=lowp)
    assert io == 0
    np.testing.assert_array_equal(po, np.arange(n))
    np.testing.assert_array_equal(LUo, LU)


@pytest.mark.parametrize("fp8", [False, True])
@pytest.mark.parametrize("b", [128, 256])
def test_lowp_factor_rounds_first_update(oracle_mod, fp8, b):
    """The first Schur update must subtract exactly q(L21) q(U12) (torch's
    roundings, scale tiles counted from the first trailing row / column):
    then the trailing block is the diagonal D and the factors are known.  The
    plain binary32 factorization of the same matrix does not give them."""
    n = b + 600
    A, LU = cf.rounded_first_update(n, b, fp8)
    LUo, po, io = oracle_mod.lu_factor_f32(A, b=b, h=128, lowp=2 if fp8 else 1)
    assert io == 0
    np.testing.assert_array_equal(po, np.arange(n))
    np.testing.assert_array_equal(LUo, LU)
    LUf, pf, _ = oracle_mod.lu_factor_f32(A, b=b, h=128)
    assert not np.array_equal(LUf, LU)


def test_rounded_update_tells_tile_origins_apart():
    """With b = 128 the step's tiles start at row / column 128; tiles counted
    from row / column 0 put other rows beside the large values, round them
    differently and leave a nonzero off-diagonal trailing block."""
    W = cf.rounded_first_update_wrong_origin(728, 128)
    off = W - np.diag(np.diag(W))
    assert np.count_nonzero(off) > 1000


def test_closed_form_exponents_match_oracle_rule(oracle_mod):
    """The tile exponents of the closed forms follow the oracle's binary32
    decision on these tiles (the exact rule and the binary32 one agree)."""
    for v in (0.4995, 0.125, 2.0 ** -15 * 1.9, 1.999, 448.0, 449.0, 3.0):
        assert cf.e4m3_exponent_exact(v) == oracle_mod.e4m3_exponent(np.float32(v))
