"""Batched factorization (one launch, one CTA per matrix) against the oracle.

Each matrix is compared with the oracle's factorization for the same panel
width (lu_batched_panel_width(n)) and leaf height 128: pivots and factors bit
for bit in binary64 and binary32.  Half of the matrices carry +n*I; those are
column diagonally dominant, a property Schur complements and row subsets
keep, so their pivots must be the identity (a closed-form pin)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu


def make_batch(sizes, seed):
    mats = []
    for i, n in enumerate(sizes):
        shift = float(n) if i % 2 == 1 else 0.0
        mats.append(wl.matrix_uniform(int(n), int(n), seed=seed, stream=i, shift=shift))
    return mats


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_matches_oracle(oracle_mod, dtype):
    torch = cuda_or_fail()
    g = lib()
    sizes = [1, 2, 15, 16, 17, 31, 33, 64, 100, 127, 128, 129, 255, 256, 257, 300, 511, 700, 1024]
    sizes += list(wl.batch_sizes(45, 16, 1024, seed=3))
    mats = make_batch(sizes, seed=11)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ndt = np.float64 if dtype == "f64" else np.float32
    dA = [torch.from_numpy(M.astype(ndt)).cuda() for M in mats]
    pivs, info = g.lu_factor_batched(dA)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    for i, (M, A, p) in enumerate(zip(mats, dA, pivs)):
        n = M.shape[0]
        b = g.batched_panel_width(n)
        if dtype == "f64":
            LUo, po, io = oracle_mod.lu_factor(M, b=b, h=128)
        else:
            LUo, po, io = oracle_mod.lu_factor_f32(M.astype(np.float32), b=b, h=128)
        assert info[i] == io, (i, n)
        np.testing.assert_array_equal(p.cpu().numpy(), po, err_msg=f"matrix {i} n={n}")
        np.testing.assert_array_equal(A.cpu().numpy(), LUo, err_msg=f"matrix {i} n={n}")
        if i % 2 == 1:
            np.testing.assert_array_equal(po, np.arange(n))


def test_batched_solve(oracle_mod):
    torch = cuda_or_fail()
    g = lib()
    sizes = [16, 40, 128, 333, 1024, 77]
    mats = make_batch(sizes, seed=5)
    dA = [torch.from_numpy(M.copy()).cuda() for M in mats]
    pivs, info = g.lu_factor_batched(dA)
    Bs = [wl.matrix_normal(M.shape[0], 1 + (i % 8), seed=9, stream=i) for i, M in enumerate(mats)]
    dB = [torch.from_numpy(B.copy()).cuda() for B in Bs]
    g.lu_solve_batched(dA, pivs, dB)
    torch.cuda.synchronize()
    for M, B, X in zip(mats, Bs, dB):
        eta = oracle_mod.backward_error(M, B, X.cpu().numpy())
        assert eta.max() <= 20 * M.shape[0] * 2.0 ** -53, eta.max()


def test_batched_rejects_out_of_range():
    torch = cuda_or_fail()
    g = lib()
    A = [torch.eye(1100, dtype=torch.float64, device="cuda"), torch.eye(8, dtype=torch.float64, device="cuda")]
    pivs, info = g.lu_factor_batched(A)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [-1, 0]
