"""Bounded device waits run out without a fault, and the library reports it.

The test hook lu_test_wait_config makes every launch at one wait site first
wait on something nothing signals (an mbarrier no thread arrives on, a solve
counter no item increments) with a short deadline.  The wait must run out
after about that deadline, the kernel must drain and exit, the call must
report LU_ETIMEOUT, and the next call with the hook off must give correct
results on the same context.  Also: the host-buffer factorization entry
point against the device one."""
import time

import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu

SHORT_NS = 50_000_000          # 50 ms


def _hooked(g, site):
    class Hook:
        def __enter__(self):
            g.set_wait_config(site, SHORT_NS, 1)

        def __exit__(self, *exc):
            g.set_wait_config(site, 0, 0)
            return False
    return Hook()


@pytest.mark.parametrize("prec", [2, 3])
def test_tcgen05_wait_runs_out_then_recovers(oracle_mod, prec):
    torch = cuda_or_fail()
    g = lib()
    rng = np.random.default_rng(3)
    M, N, K = 700, 520, 128
    L = rng.standard_normal((M, K)).astype(np.float32)
    U = rng.standard_normal((K, N)).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    dL, dU = torch.from_numpy(L).cuda(), torch.from_numpy(U).cuda()
    with _hooked(g, g.LU_WAIT_SITE_TC):
        dC = torch.from_numpy(C.copy()).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = g.lu_gemm_lowp(dL, dU, dC, precision=prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    assert int(st.cpu()[0]) == -g.LU_ETIMEOUT
    assert 0.04 <= dt < 3.0, dt                      # the deadline, not the 4 s default
    dC = torch.from_numpy(C.copy()).cuda()
    _, st = g.lu_gemm_lowp(dL, dU, dC, precision=prec)
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == 0
    Cref, Sabs = oracle_mod.gemm_lowp(L, U, C, fp8=(prec == 3))
    err = np.abs(dC.cpu().numpy().astype(np.float64) - Cref)
    assert (err <= 2.0 ** -22 * np.abs(Cref) + (K + 2) * 2.0 ** -21 * Sabs + 1e-30).all()


def test_mixed_factor_reports_timeout_in_info(oracle_mod):
    """The bf16 factorization hands the tcgen05 status to info: -LU_ETIMEOUT."""
    torch = cuda_or_fail()
    g = lib()
    n = 512
    A = wl.matrix_uniform(n, n, seed=4).astype(np.float32)
    with _hooked(g, g.LU_WAIT_SITE_TC):
        dA = torch.from_numpy(A.copy()).cuda()
        piv, info = g.lu_factor_f32(dA, b=128, h=128, precision=g.LU_PREC_BF16)
        torch.cuda.synchronize()
    assert int(info.cpu()[0]) == -g.LU_ETIMEOUT
    dA = torch.from_numpy(A.copy()).cuda()
    piv, info = g.lu_factor_f32(dA, b=128, h=128, precision=g.LU_PREC_BF16)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    _, po, _ = oracle_mod.lu_factor_f32(A, b=128, h=128, lowp=1)
    np.testing.assert_array_equal(piv.cpu().numpy()[:128], po[:128])


def test_solve_wait_runs_out_then_recovers(oracle_mod):
    torch = cuda_or_fail()
    g = lib()
    n, nrhs = 900, 3
    A = wl.matrix_uniform(n, n, seed=6)
    B = wl.matrix_uniform(n, nrhs, seed=6, stream=1)
    LU, piv, info = oracle_mod.lu_factor(A, b=64, h=128)
    dLU = torch.from_numpy(LU).cuda()
    dpiv = torch.from_numpy(piv.astype(np.int32)).cuda()
    with _hooked(g, g.LU_WAIT_SITE_SOLVE):
        dB = torch.from_numpy(B.copy()).cuda()
        t0 = time.perf_counter()
        with pytest.raises(g.LuError) as exc:
            g.lu_solve(dLU, dpiv, dB)
        dt = time.perf_counter() - t0
    assert exc.value.code == g.LU_ETIMEOUT
    assert 0.04 <= dt < 3.0, dt
    dB = torch.from_numpy(B.copy()).cuda()
    g.lu_solve(dLU, dpiv, dB)
    torch.cuda.synchronize()
    X = dB.cpu().numpy()
    assert oracle_mod.backward_error(A, B, X).max() <= 20 * n * 2.0 ** -53


def test_ir_solve_passes_the_timeout_up():
    torch = cuda_or_fail()
    g = lib()
    n = 600
    A = torch.from_numpy(wl.matrix_uniform(n, n, seed=8, shift=float(n))).cuda()
    B = torch.ones(n, 2, dtype=torch.float64, device="cuda")
    with _hooked(g, g.LU_WAIT_SITE_SOLVE):
        with pytest.raises(g.LuError) as exc:
            g.ir_solve(A, B, precision=g.LU_PREC_BF16)
    assert exc.value.code == g.LU_ETIMEOUT
    X, res = g.ir_solve(A, B, precision=g.LU_PREC_BF16)
    assert res["eta"] <= 1e-12


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("m,n,lda,b", [(700, 700, 710, 64), (640, 640, 640, 64), (1500, 1200, 1200, 128),
                                        (300, 500, 503, 32)])
def test_host_factor_equals_device_factor(m, n, lda, b, pinned):
    """lu_factor_host (host buffers, copies inside the call) returns the
    device factorization's L\\U, pivots and info bit for bit."""
    torch = cuda_or_fail()
    g = lib()
    A = wl.matrix_normal(m, n, seed=m + n)
    dA = torch.from_numpy(A.copy()).cuda()
    dpiv, dinfo = g.lu_factor_ex(dA, b=b, h=128)
    torch.cuda.synchronize()
    buf = torch.full((m, lda), float("nan"), dtype=torch.float64)
    if pinned:
        buf = buf.pin_memory()
    buf[:, :n] = torch.from_numpy(A)
    hv = buf[:, :n]
    piv, info = g.lu_factor_host(hv, b=b, h=128)
    assert info == int(dinfo.cpu()[0]) == 0
    np.testing.assert_array_equal(piv.numpy(), dpiv.cpu().numpy())
    np.testing.assert_array_equal(hv.numpy(), dA.cpu().numpy())
    assert torch.isnan(buf[:, n:]).all()              # the padding is not touched
