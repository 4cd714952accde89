"""Closed forms for the mixed-precision factorization (binary32 panel, Schur
update with bfloat16 / fp8-e4m3 operands, one power-of-two scale per 256 x 256
operand tile counted from the step's first trailing row / column, fp32
accumulation).

Two constructions, both with P = I and factors known in advance:

* ``exact_factors``: A = L U with every entry of L and U exactly
  representable in bf16 and in e4m3 under any scale the tile rule can pick,
  and every partial sum of every element exactly representable in binary32.
  Every step of the factorization is then exact, so the factors come back as
  L and U bit for bit in either low-precision mode.  Row classes of L and
  column classes of U differ in magnitude by 4x or more, so an operand value
  scaled with another tile's exponent saturates at 448 and the result moves.

* ``rounded_first_update``: A = [[L00 U00, L00 U12], [L21 U00, q(L21) q(U12) + D]]
  where L21 and U12 carry more significant bits than the low-precision format
  and q() is the format's rounding with the tile scales of the first step.
  After that step the trailing block is exactly the diagonal D, so the
  factors are L = [[L00, 0], [L21, I]] and U = [[U00, U12], [0, D]] -- but only
  if the first update subtracted exactly q(L21) q(U12): no rounding, another
  rounding, another tile origin or another scale rule leaves a nonzero
  off-diagonal trailing block.  Some rows of L21 (and columns of U12) are
  2^-14 smaller than the rest; in e4m3 they round onto the subnormal grid when
  their tile also holds large values, and keep four significant bits in a
  tile of their own, so the tile origin decides the result.

The roundings here are torch's float -> bfloat16 / float8_e4m3fn conversions
(round to nearest, ties to even), which neither the oracle nor the CUDA
library uses.  Every builder asserts the exactness it relies on: each product
and each subset sum of an element's update terms must be exactly
representable in binary32 (a sum of terms on a grid 2^g whose absolute sum is
below 2^(24+g) is), so the result does not depend on summation order.
"""
from __future__ import annotations

import numpy as np

import workloads as wl

E4M3_MAX = 448.0
SCALE_TILE = 256


def _u(seed, stream, shape):
    cnt = int(np.prod(shape))
    return wl.uniform01(seed, stream, np.arange(cnt, dtype=np.uint64)).reshape(shape)


def _pick(u, values):
    """Map uniforms in [0,1) onto a value list."""
    v = np.asarray(values, dtype=np.float64)
    return v[np.minimum((u * len(v)).astype(np.int64), len(v) - 1)]


def _lsb_exp(x):
    """Exponent g of the lowest set bit of each nonzero |x| (x = odd * 2^g);
    +inf where x == 0."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    m, e = np.frexp(x)
    mi = (m * 2.0 ** 53).astype(np.int64)
    low = mi & (-mi)
    out = np.full(x.shape, np.inf)
    nz = mi != 0
    out[nz] = np.log2(low[nz].astype(np.float64)) + e[nz] - 53
    return out


def assert_sums_exact_f32(Lm, Um, rows=64):
    """Every subset sum of the terms Lm[i,p] Um[p,j] (over p) is exactly
    representable in binary32 for every (i, j)."""
    gl = _lsb_exp(Lm)
    gu = _lsb_exp(Um)
    Sabs = np.abs(Lm) @ np.abs(Um)
    for r0 in range(0, Lm.shape[0], rows):
        g = np.min(gl[r0:r0 + rows, :, None] + gu[None, :, :], axis=1)
        s = Sabs[r0:r0 + rows]
        live = np.isfinite(g)
        assert np.all(s[live] < 2.0 ** (24 + g[live])), "closed form not exact in binary32"
    # products themselves: at most 24 significant bits
    return Sabs


def e4m3_exponent_exact(maxabs: float) -> int:
    """Smallest e with maxabs * 2^-e <= 448 (0 for an all-zero tile)."""
    if maxabs <= 0.0:
        return 0
    e = -200
    while np.ldexp(maxabs, -e) > E4M3_MAX:
        e += 1
    while e > -200 and np.ldexp(maxabs, -(e - 1)) <= E4M3_MAX:
        e -= 1
    return e


def quantize(X, fp8: bool, axis: int):
    """q(X) as float64: bf16 (scale 1), or e4m3 with one power-of-two scale per
    256 rows (axis 0, the L21 operand) or 256 columns (axis 1, U12), counted
    from index 0 of X.  Returns (qX, exponents)."""
    import torch
    X = np.asarray(X, dtype=np.float32)
    if not fp8:
        q = torch.from_numpy(X.copy()).to(torch.bfloat16).to(torch.float64).numpy()
        return q, []
    out = np.empty(X.shape, dtype=np.float64)
    exps = []
    n = X.shape[axis]
    for t0 in range(0, n, SCALE_TILE):
        sl = (slice(t0, t0 + SCALE_TILE), slice(None)) if axis == 0 else (slice(None), slice(t0, t0 + SCALE_TILE))
        blk = X[sl].astype(np.float64)
        e = e4m3_exponent_exact(float(np.abs(blk).max()) if blk.size else 0.0)
        exps.append(e)
        scaled = torch.from_numpy(np.ldexp(blk, -e).astype(np.float32))
        q = scaled.to(torch.float8_e4m3fn).to(torch.float64).numpy()
        out[sl] = np.ldexp(q, e)
    return out, exps


def _combine(L, U):
    n = L.shape[0]
    return np.tril(L, -1) + np.triu(U)


def exact_factors(n: int, seed: int = 5):
    """(A, LU) with A = L U exact in binary32, every step of any blocked
    factorization of A exact, and both operands of every low-precision update
    exactly representable in bf16 and in e4m3 under their own tile's scale.
    LU holds L (strict lower) and U (upper) as binary32."""
    i = np.arange(n)
    big_row = (i // 160) % 3 == 0                 # L rows with |l| up to 1/2
    big_col = (i // 384) % 2 == 1                 # U columns with |u| up to 3
    u = _u(seed, 60, (4, n, n))
    l_big = _pick(u[0], [0, 0, 0, 0, 0.25, -0.25, 0.375, -0.375, 0.5, -0.5])
    l_small = _pick(u[0], [0, 0, 0, 0, 0.0625, -0.0625, 0.09375, -0.09375, 0.125, -0.125])
    L = np.where(big_row[:, None], l_big, l_small)
    L = np.tril(L, -1) + np.eye(n)
    u_big = _pick(u[1], [0, 0, 0, 0, 1.0, -1.0, 1.5, -1.5, 2.0, -2.0, 3.0, -3.0])
    u_small = _pick(u[1], [0, 0, 0, 0, 0.125, -0.125, 0.1875, -0.1875, 0.25, -0.25])
    U = np.where(big_col[None, :], u_big, u_small)
    diag = _pick(u[2][0], [1.0, -1.0, 1.5, -1.5, 2.0, -2.0])
    U = np.triu(U, 1) + np.diag(diag)
    assert_sums_exact_f32(L, U)
    A = L @ U
    A32 = A.astype(np.float32)
    assert np.array_equal(A32.astype(np.float64), A)
    return A32, _combine(L, U).astype(np.float32)


def rounded_first_update(n: int, b: int, fp8: bool, seed: int = 9):
    """(A, LU) for the construction with a rounded first Schur update (see the
    module docstring).  Rows of L21 / columns of U12 of the trailing block are
    arranged in 128-row bands so that, with b = 128, a band of tiny values
    shares a scale tile with large values under the step-relative origin but
    not under an origin at row / column 0 of the matrix."""
    M = n - b
    assert M > 0
    u = _u(seed + (1 if fp8 else 0), 70, (8, n, n))
    # L00 unit lower, U00 upper, small dyadic entries
    L00 = np.tril(_pick(u[0][:b, :b], [0, 0, 0, 0, 0, 0.25, -0.25, 0.5, -0.5]), -1) + np.eye(b)
    U00 = np.triu(_pick(u[1][:b, :b], [0, 0, 0, 0, 0, 0.5, -0.5, 1.0, -1.0]), 1) + \
        np.diag(_pick(u[2][0, :b], [1.0, -1.0, 2.0, -2.0]))
    # trailing rows / columns in bands of 128: pattern big, tiny, big, tiny, tiny
    band = (np.arange(M) + b) // 128
    tiny = np.isin(band % 5, [1, 3, 4])
    # L21: sparse, 12 significant bits, |l| in [1/8, 1/2) (tiny rows: * 2^-14)
    mant = np.floor(1024 + u[3][:M, :b] * 3072)                    # [1024, 4096)
    sgn = np.where(u[4][:M, :b] < 0.5, -1.0, 1.0)
    keep = u[5][:M, :b] < 0.125
    L21 = np.where(keep, sgn * mant * 2.0 ** -13, 0.0)
    L21[tiny] *= 2.0 ** -14
    # U12: sparse, 12 significant bits, |u| in [1/2, 2) (tiny columns: * 2^-14)
    mant = np.floor(2048 + u[3][M:M + b, :M] * 6144)               # [2048, 8192)
    sgn = np.where(u[6][:b, :M] < 0.5, -1.0, 1.0)
    keep = u[7][:b, :M] < 0.125
    U12 = np.where(keep, sgn * mant * 2.0 ** -12, 0.0)
    U12[:, tiny] *= 2.0 ** -14
    # no update term on the diagonal of a tiny row (its sum would span more
    # bits than binary32 holds once D is added)
    for i in np.nonzero(tiny)[0]:
        U12[L21[i] != 0, i] = 0.0
    # the step's rounded operands (tiles counted from the first trailing row / column)
    qL, _ = quantize(L21, fp8, axis=0)
    qU, _ = quantize(U12, fp8, axis=1)
    assert not np.array_equal(qL, L21) and not np.array_equal(qU, U12)
    # D: +-1 or +-2 on the diagonal
    d = _pick(u[2][1, :M], [1.0, -1.0, 2.0, -2.0])
    acc_abs = assert_sums_exact_f32(qL, qU)
    acc = qL @ qU
    A11 = acc + np.diag(d)
    for Lm, Um in ((L00, U00), (L21, U00), (L00, U12)):
        assert_sums_exact_f32(Lm, Um)
    A = np.block([[L00 @ U00, L00 @ U12], [L21 @ U00, A11]])
    A32 = A.astype(np.float32)
    assert np.array_equal(A32.astype(np.float64), A), "closed form not representable in binary32"
    assert acc_abs.max() > 0
    LU = np.block([[_combine(L00, U00), U12], [L21, np.diag(d)]]).astype(np.float32)
    assert np.array_equal(LU.astype(np.float64), np.block([[_combine(L00, U00), U12], [L21, np.diag(d)]]))
    return A32, LU


def rounded_first_update_wrong_origin(n: int, b: int, seed: int = 9):
    """The trailing block that an e4m3 update with scale tiles counted from
    row / column 0 of the matrix (instead of the step's first trailing row /
    column) would leave after the first step of ``rounded_first_update``'s
    matrix: the check that the construction can tell the two origins apart."""
    A, LU = rounded_first_update(n, b, True, seed)
    M = n - b
    L21 = LU[b:, :b].astype(np.float64)
    U12 = LU[:b, b:].astype(np.float64)
    pad = b % SCALE_TILE
    Lp = np.vstack([np.zeros((pad, b)), L21])
    Up = np.hstack([np.zeros((b, pad)), U12])
    qL, _ = quantize(Lp, True, axis=0)
    qU, _ = quantize(Up, True, axis=1)
    return A[b:, b:].astype(np.float64) - qL[pad:] @ qU[:, pad:]
