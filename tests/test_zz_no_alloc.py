"""lu_residual_noalloc: the residual and backward error for callers that
cannot allocate device memory while they run (its scratch is a fixed array
inside the library).  Checked through the C ABI against lu_residual on two
calls in a row, so that a second call does not read the first one's leftovers.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu


def _entry():
    lib()
    from paper_2010_05975_gb300 import _native as nat
    L = nat.library()
    P, I = ctypes.c_void_p, ctypes.c_int
    for name in ("lu_residual", "lu_residual_noalloc"):
        fn = getattr(L, name)
        fn.argtypes = [I, I, P, I, P, I, P, I, P, I, P, P]
        fn.restype = I
    return L


def _call(fn, A, X, B, torch):
    n, nr = X.shape
    R = torch.full((n, nr), float("nan"), dtype=torch.float64, device="cuda")
    eta = torch.full((nr,), float("nan"), dtype=torch.float64, device="cuda")
    rc = fn(n, nr, A.data_ptr(), n, X.data_ptr(), nr, B.data_ptr(), nr, R.data_ptr(), nr, eta.data_ptr(),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, R.cpu().numpy(), eta.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    torch = cuda_or_fail()
    L = _entry()
    cases = [(700, 16, 1), (1500, 5, 2)]          # two calls in a row, different shapes
    for n, nr, seed in cases:
        A = torch.from_numpy(wl.matrix_uniform(n, n, seed=seed)).cuda()
        X = torch.from_numpy(wl.matrix_normal(n, nr, seed=seed + 10)).cuda()
        B = torch.from_numpy(wl.matrix_normal(n, nr, seed=seed + 20)).cuda()
        rc0, R0, e0 = _call(L.lu_residual, A, X, B, torch)
        rc1, R1, e1 = _call(L.lu_residual_noalloc, A, X, B, torch)
        assert rc0 == 0 and rc1 == 0
        scale = np.abs(A.cpu().numpy()).sum(axis=1).max() * np.abs(X.cpu().numpy()).max()
        assert np.abs(R1 - R0).max() <= 4 * n * 2.0 ** -53 * scale
        np.testing.assert_allclose(e1, e0, rtol=1e-12)
        assert np.isfinite(e1).all()


def test_noalloc_rejects_too_many_rhs():
    torch = cuda_or_fail()
    L = _entry()
    n, nr = 64, 65
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    X = torch.zeros((n, nr), dtype=torch.float64, device="cuda")
    rc, R, e = _call(L.lu_residual_noalloc, A, X, X, torch)
    assert rc == -2
    assert np.isnan(R).all() and np.isnan(e).all()
