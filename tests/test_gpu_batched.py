"""Batched factorization (one launch, one CTA per matrix) against the oracle.

Each matrix is compared with the oracle's factorization for the same panel
width (lu_batched_panel_width_dt(n, dtype)) and leaf height 128: pivots and factors bit
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
        b = g.batched_panel_width(n, tdt)
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


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_every_panel_width_matches_oracle(oracle_mod, dtype):
    """The tuning sweep's widths (8, 16, 32 for every size class) keep the
    oracle's factors bit for bit; the table is restored afterwards."""
    torch = cuda_or_fail()
    g = lib()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ndt = np.float64 if dtype == "f64" else np.float32
    sizes = [5, 40, 100, 200, 300, 600]
    mats = make_batch(sizes, seed=21)
    try:
        for b in (8, 16, 32):
            g.set_batched_panel_widths(tdt, [b] * 6)
            dA = [torch.from_numpy(M.astype(ndt)).cuda() for M in mats]
            pivs, info = g.lu_factor_batched(dA)
            torch.cuda.synchronize()
            for M, A, p in zip(mats, dA, pivs):
                assert g.batched_panel_width(M.shape[0], tdt) == b
                if dtype == "f64":
                    LUo, po, io = oracle_mod.lu_factor(M, b=b, h=128)
                else:
                    LUo, po, io = oracle_mod.lu_factor_f32(M.astype(np.float32), b=b, h=128)
                np.testing.assert_array_equal(p.cpu().numpy(), po)
                np.testing.assert_array_equal(A.cpu().numpy(), LUo)
    finally:
        g.set_batched_panel_widths(tdt, None)


def test_batched_factor_and_solve_replay_in_a_cuda_graph(oracle_mod):
    """lu_factor_batched + lu_solve_batched captured in one CUDA graph and
    replayed twice give the direct calls' results bit for bit."""
    torch = cuda_or_fail()
    g = lib()
    sizes = [16, 40, 128, 333, 1024, 77, 250]
    mats = make_batch(sizes, seed=31)
    Bs = [wl.matrix_normal(M.shape[0], 1 + (i % 8), seed=4, stream=i) for i, M in enumerate(mats)]
    # direct calls
    dA = [torch.from_numpy(M.copy()).cuda() for M in mats]
    dB = [torch.from_numpy(B.copy()).cuda() for B in Bs]
    pivs, info = g.lu_factor_batched(dA)
    g.lu_solve_batched(dA, pivs, dB)
    torch.cuda.synchronize()
    # the same work as one graph
    gr = g.BatchedFactorSolve([torch.from_numpy(M.copy()).cuda() for M in mats],
                              [torch.from_numpy(B.copy()).cuda() for B in Bs]).capture()
    for _ in range(2):
        for a in gr.A:
            a.fill_(float("nan"))          # the replay must restore the inputs itself
        torch.cuda.synchronize()
        gr.replay()
        torch.cuda.synchronize()
        for a1, a2, b1, b2 in zip(dA, gr.A, dB, gr.B):
            np.testing.assert_array_equal(a1.cpu().numpy(), a2.cpu().numpy())
            np.testing.assert_array_equal(b1.cpu().numpy(), b2.cpu().numpy())
