"""lu_residual_noalloc: the residual and backward error for callers that
cannot allocate device memory while they run -- a serving loop that reserves
all of its memory before it takes requests, or a process whose GPU memory
another framework's caching allocator owns.  Its scratch is a fixed array
inside the library.

Checked through the C ABI on two calls in a row (so that a second call does
not read the first one's leftovers): against the host's binary64 B - AX, the
oracle's backward error and the allocating entry point lu_residual; and the
calls must leave the device's stream-ordered pool and free memory untouched.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values (cuda.h)
_USED_MEM_CURRENT = 7
_USED_MEM_HIGH = 8


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


class Pool:
    """Read-only view of a stream-ordered memory pool through the driver API:
    the current device's default pool (what cudaMallocAsync draws from), or
    the library's own pool (lu_memory_pool, where its workspace comes from)."""

    def __init__(self, torch, library=None):
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.pool = ctypes.c_void_p(0)
        if library is None:
            dev = ctypes.c_int(0)
            assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
            assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0
        else:
            library.lu_memory_pool.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
            assert library.lu_memory_pool(ctypes.byref(self.pool)) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _call(fn, A, X, B, torch):
    n, nr = X.shape
    R = torch.full((n, nr), float("nan"), dtype=torch.float64, device="cuda")
    eta = torch.full((nr,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = fn(n, nr, A.data_ptr(), n, X.data_ptr(), nr, B.data_ptr(), nr, R.data_ptr(), nr, eta.data_ptr(),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, R.cpu().numpy(), eta.cpu().numpy()


def test_noalloc_matches_host_residual_and_oracle_twice(oracle_mod):
    torch = cuda_or_fail()
    L = _entry()
    cases = [(700, 16, 1), (1500, 5, 2), (300, 64, 3)]      # calls in a row, different shapes
    for n, nr, seed in cases:
        An = wl.matrix_uniform(n, n, seed=seed)
        Xn = wl.matrix_normal(n, nr, seed=seed + 10)
        Bn = wl.matrix_normal(n, nr, seed=seed + 20)
        A, X, B = (torch.from_numpy(M).cuda() for M in (An, Xn, Bn))
        rc1, R1, e1 = _call(L.lu_residual_noalloc, A, X, B, torch)
        assert rc1 == 0
        # the host's binary64 residual: |R - (B - AX)| within n roundings of |A||X| + |B|
        Rh = Bn - An @ Xn
        bound = 4 * n * 2.0 ** -53 * (np.abs(An) @ np.abs(Xn) + np.abs(Bn))
        assert (np.abs(R1 - Rh) <= bound).all()
        # the oracle's normwise backward error, column by column
        eo = oracle_mod.backward_error(An, Bn, Xn)
        np.testing.assert_allclose(e1, eo, rtol=1e-10, atol=0)
        # and the allocating entry point
        rc0, R0, e0 = _call(L.lu_residual, A, X, B, torch)
        assert rc0 == 0
        assert (np.abs(R1 - R0) <= bound).all()
        np.testing.assert_allclose(e1, e0, rtol=1e-12)


def test_noalloc_allocates_nothing():
    """Around a call (after a first one, which may load the library's device
    code), the used-memory high watermarks of the default pool and of the
    library's pool stay where they were and the device's free memory does not
    change; the same measurement around lu_residual does see its workspace
    allocation in the library's pool."""
    torch = cuda_or_fail()
    L = _entry()
    dpool = Pool(torch)
    pool = Pool(torch, L)
    n, nr = 1000, 12
    A = torch.from_numpy(wl.matrix_uniform(n, n, seed=7)).cuda()
    X = torch.from_numpy(wl.matrix_normal(n, nr, seed=8)).cuda()
    B = torch.from_numpy(wl.matrix_normal(n, nr, seed=9)).cuda()
    assert _call(L.lu_residual_noalloc, A, X, B, torch)[0] == 0
    R = torch.empty((n, nr), dtype=torch.float64, device="cuda")
    eta = torch.empty(nr, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def measured(fn, p):
        torch.cuda.synchronize()
        p.reset_high()
        used0 = p.get(_USED_MEM_CURRENT)
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            assert fn(n, nr, A.data_ptr(), n, X.data_ptr(), nr, B.data_ptr(), nr, R.data_ptr(), nr,
                      eta.data_ptr(), s) == 0
        torch.cuda.synchronize()
        return used0, p.get(_USED_MEM_HIGH), free0, torch.cuda.mem_get_info()[0]

    for p in (dpool, pool):
        used0, high, free0, free1 = measured(L.lu_residual_noalloc, p)
        assert high == used0
        assert free1 == free0
    used0, high, _, _ = measured(L.lu_residual, pool)
    assert high > used0                      # the check sees a stream-ordered allocation


def test_noalloc_rejects_too_many_rhs():
    torch = cuda_or_fail()
    L = _entry()
    n, nr = 64, 65
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    X = torch.zeros((n, nr), dtype=torch.float64, device="cuda")
    rc, R, e = _call(L.lu_residual_noalloc, A, X, X, torch)
    assert rc == -2
    assert np.isnan(R).all() and np.isnan(e).all()
