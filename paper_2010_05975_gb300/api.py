"""Python face of the C ABI: same names, torch tensors in, raw pointers out."""
from __future__ import annotations

import ctypes

import torch

from . import _native as nat


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require(t: torch.Tensor, name: str, dtype, ndim: int):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    if ndim == 2 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major with unit column stride")


def lu_factor(A: torch.Tensor, piv: torch.Tensor | None = None, info: torch.Tensor | None = None,
              stream=None):
    """In-place PA = LU of a square float64 CUDA tensor.  Returns (piv, info)
    as int32 CUDA tensors (piv 0-based LAPACK style); nothing is synchronised."""
    _require(A, "A", torch.float64, 2)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("lu_factor needs a square matrix; use lu_factor_ex")
    if piv is None:
        piv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    lib = nat.library()
    rc = lib.lu_factor(n, A.data_ptr(), max(A.stride(0), 1), piv.data_ptr(), info.data_ptr(),
                       _stream_handle(stream))
    nat.check("lu_factor", rc)
    return piv[:n], info


def lu_factor_ex(A: torch.Tensor, b: int = 0, h: int = 0, precision: int = nat.LU_PREC_F64,
                 piv: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None):
    """In-place m x n factorization with panel width b and leaf height h."""
    _require(A, "A", torch.float64, 2)
    m, n = A.shape
    k = min(m, n)
    if piv is None:
        piv = torch.empty(max(k, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    opts = nat.lu_opts(b, h, precision)
    lib = nat.library()
    rc = lib.lu_factor_ex(m, n, A.data_ptr(), max(A.stride(0), 1), piv.data_ptr(), info.data_ptr(),
                          ctypes.byref(opts), _stream_handle(stream))
    nat.check("lu_factor_ex", rc)
    return piv[:k], info


def lu_solve(LU: torch.Tensor, piv: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """Overwrite B (n or n x nrhs, float64, CUDA) with the solution of A X = B."""
    _require(LU, "LU", torch.float64, 2)
    n = LU.shape[0]
    B2 = B if B.dim() == 2 else B.view(n, 1)
    _require(B2, "B", torch.float64, 2)
    lib = nat.library()
    rc = lib.lu_solve(n, B2.shape[1], LU.data_ptr(), max(LU.stride(0), 1), piv.data_ptr(), B2.data_ptr(),
                      max(B2.stride(0), 1), _stream_handle(stream))
    nat.check("lu_solve", rc)
    return B


def prof_begin() -> None:
    nat.check("lu_prof_begin", nat.library().lu_prof_begin())


def prof_end() -> dict:
    """Close a profiling session; returns {class: {launches, ms, flops, bytes}}."""
    arr = (nat.lu_prof_entry * 16)()
    n = ctypes.c_int(0)
    nat.check("lu_prof_end", nat.library().lu_prof_end(arr, 16, ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        e = arr[i]
        out[nat.PROF_CLASSES[e.kernel_class]] = {"launches": e.launches, "ms": e.total_ms,
                                                 "flops": e.total_flops, "bytes": e.total_bytes}
    return out


def kernel_launch_count() -> int:
    return int(nat.library().lu_kernel_launch_count())


def lu_factor_host(A_host: torch.Tensor, b: int = 0, h: int = 0, piv: torch.Tensor | None = None,
                   stream=None):
    """In-place factorization of a matrix in host memory through the C ABI's
    lu_factor_host (copy in, factor on the device, copy L\\U and the pivots
    back; returns when they are in host memory).  A_host is a row-major
    float64 CPU tensor, overwritten by L and U; page-locked memory
    (pin_memory()) makes the copies run at the link's rate.  Returns
    (piv, info) with piv an int32 CPU tensor."""
    if A_host.is_cuda or A_host.dtype != torch.float64 or A_host.dim() != 2 or A_host.stride(1) != 1:
        raise TypeError("A_host must be a row-major 2-D float64 CPU tensor")
    m, n = A_host.shape
    k = min(m, n)
    if piv is None:
        piv = torch.empty(max(k, 1), dtype=torch.int32, pin_memory=A_host.is_pinned())
    info = ctypes.c_int(0)
    opts = nat.lu_opts(b, h, nat.LU_PREC_F64)
    rc = nat.library().lu_factor_host(m, n, A_host.data_ptr(), max(A_host.stride(0), 1), piv.data_ptr(),
                                      ctypes.byref(info), ctypes.byref(opts), _stream_handle(stream))
    nat.check("lu_factor_host", rc)
    return piv[:k], info.value


def set_wait_config(site: int, wait_ns: int = 0, inject: int = 0) -> None:
    """Test hook: deadline of one wait site's dependency waits (0 = the 4 s
    default) and whether launches there first wait on something never
    signalled, so that the wait runs out (see lu_test_wait_config)."""
    nat.check("lu_test_wait_config", nat.library().lu_test_wait_config(int(site), int(wait_ns), int(inject)))


def lu_factor_f32(A: torch.Tensor, b: int = 0, h: int = 0, precision: int = nat.LU_PREC_F32,
                  piv: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None,
                  defer: int = 0):
    """In-place factorization of a float32 CUDA matrix.  precision selects the
    Schur-update operands: F32, BF16 or FP8 (tensor cores); defer (BF16 / FP8
    only) how many panels' trailing updates one pass applies (0 = default)."""
    _require(A, "A", torch.float32, 2)
    m, n = A.shape
    k = min(m, n)
    if piv is None:
        piv = torch.empty(max(k, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    opts = nat.lu_opts(b, h, precision, defer)
    rc = nat.library().lu_factor_f32(m, n, A.data_ptr(), max(A.stride(0), 1), piv.data_ptr(), info.data_ptr(),
                                     ctypes.byref(opts), _stream_handle(stream))
    nat.check("lu_factor_f32", rc)
    return piv[:k], info


def chol_factor(A: torch.Tensor, b: int = 0, info: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """In-place Cholesky A = L L^T of a square float64 or float32 CUDA matrix
    (lower triangle read and overwritten with L; strict upper untouched).
    Returns info (int32 CUDA tensor, 0 or the first non-positive pivot's
    column + 1); nothing is synchronised."""
    if not isinstance(A, torch.Tensor) or A.dtype not in (torch.float64, torch.float32):
        raise TypeError("A must be a float64 or float32 CUDA tensor")
    _require(A, "A", A.dtype, 2)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("chol_factor needs a square matrix")
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    opts = nat.lu_opts(b, 0, 0)
    lib = nat.library()
    fn, name = (lib.chol_factor, "chol_factor") if A.dtype == torch.float64 else \
        (lib.chol_factor_f32, "chol_factor_f32")
    rc = fn(n, A.data_ptr(), max(A.stride(0), 1), info.data_ptr(), ctypes.byref(opts), _stream_handle(stream))
    nat.check(name, rc)
    return info


def chol_solve(L: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """Overwrite B (n or n x nrhs, L's dtype, CUDA) with the solution of
    L L^T X = B, L the lower triangle of chol_factor's result."""
    if not isinstance(L, torch.Tensor) or L.dtype not in (torch.float64, torch.float32):
        raise TypeError("L must be a float64 or float32 CUDA tensor")
    _require(L, "L", L.dtype, 2)
    n = L.shape[0]
    Bm = B.view(n, 1) if B.dim() == 1 else B
    _require(Bm, "B", L.dtype, 2)
    lib = nat.library()
    fn, name = (lib.chol_solve, "chol_solve") if L.dtype == torch.float64 else (lib.chol_solve_f32, "chol_solve_f32")
    rc = fn(n, Bm.shape[1], L.data_ptr(), max(L.stride(0), 1), Bm.data_ptr(), max(Bm.stride(0), 1),
            _stream_handle(stream))
    nat.check(name, rc)
    return B


def lu_solve_f32(LU: torch.Tensor, piv: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    _require(LU, "LU", torch.float32, 2)
    n = LU.shape[0]
    B2 = B if B.dim() == 2 else B.view(n, 1)
    _require(B2, "B", torch.float32, 2)
    rc = nat.library().lu_solve_f32(n, B2.shape[1], LU.data_ptr(), max(LU.stride(0), 1), piv.data_ptr(),
                                    B2.data_ptr(), max(B2.stride(0), 1), _stream_handle(stream))
    nat.check("lu_solve_f32", rc)
    return B


def lu_gemm_lowp(L: torch.Tensor, U: torch.Tensor, C: torch.Tensor, precision: int = nat.LU_PREC_BF16,
                 status: torch.Tensor | None = None, stream=None):
    """C -= sL sU round(L/sL) round(U/sU) on the tensor cores (float32 in/out)."""
    for t, nm in ((L, "L"), (U, "U"), (C, "C")):
        _require(t, nm, torch.float32, 2)
    M, K = L.shape
    N = U.shape[1]
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=C.device)
    rc = nat.library().lu_gemm_lowp(M, N, K, L.data_ptr(), max(L.stride(0), 1), U.data_ptr(), max(U.stride(0), 1),
                                    C.data_ptr(), max(C.stride(0), 1), precision, status.data_ptr(),
                                    _stream_handle(stream))
    nat.check("lu_gemm_lowp", rc)
    return C, status


def lu_residual(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor, R: torch.Tensor | None = None,
                eta: torch.Tensor | None = None, stream=None):
    """R = B - A X (float64) and eta per column."""
    _require(A, "A", torch.float64, 2)
    n = A.shape[0]
    X2 = X if X.dim() == 2 else X.view(n, 1)
    B2 = B if B.dim() == 2 else B.view(n, 1)
    nr = X2.shape[1]
    if R is None:
        R = torch.empty((n, nr), dtype=torch.float64, device=A.device)
    if eta is None:
        eta = torch.empty(nr, dtype=torch.float64, device=A.device)
    rc = nat.library().lu_residual(n, nr, A.data_ptr(), max(A.stride(0), 1), X2.data_ptr(), max(X2.stride(0), 1),
                                   B2.data_ptr(), max(B2.stride(0), 1), R.data_ptr(), max(R.stride(0), 1),
                                   eta.data_ptr(), _stream_handle(stream))
    nat.check("lu_residual", rc)
    return R, eta


def ir_solve(A: torch.Tensor, B: torch.Tensor, X: torch.Tensor | None = None, precision: int = nat.LU_PREC_BF16,
             tol: float = 1e-12, b: int = 0, h: int = 0, max_iter: int = 0, gmres_restart: int = 0,
             krylov_products: int = 0, inner_steps: int = 0, stream=None):
    """Solve A X = B (float64 CUDA tensors) with a low-precision factorization
    and float64 refinement.  krylov_products: 0 adaptive (binary32 multiplies
    first), 1 binary64 only, 2 binary32 multiplies only.  inner_steps:
    binary32-product inner steps per classical step (0 default, < 0 none).
    Synchronizes the stream; returns (X, result)."""
    _require(A, "A", torch.float64, 2)
    n = A.shape[0]
    B2 = B if B.dim() == 2 else B.view(n, 1)
    _require(B2, "B", torch.float64, 2)
    if X is None:
        X = torch.empty_like(B2)
    X2 = X if X.dim() == 2 else X.view(n, 1)
    opts = nat.ir_opts(precision, b, h, tol, max_iter, gmres_restart, krylov_products, inner_steps)
    res = nat.ir_result()
    rc = nat.library().ir_solve(n, B2.shape[1], A.data_ptr(), max(A.stride(0), 1), B2.data_ptr(),
                                max(B2.stride(0), 1), X2.data_ptr(), max(X2.stride(0), 1), ctypes.byref(opts),
                                ctypes.byref(res), _stream_handle(stream))
    nat.check("ir_solve", rc)
    out = {"iters": res.iters, "gmres_iters": res.gmres_iters, "path": res.path, "info": res.info,
           "eta": res.eta, "eta0": res.eta0, "precision": res.precision, "refactors": res.refactors,
           "cycles32": res.cycles32, "cycles64": res.cycles64, "inner_steps": res.inner_steps}
    return X, out


def _keep_for_stream(stream, *tensors):
    """The size and pointer arrays are made on the current stream and freed
    when this call returns; the caching allocator hands their memory out again
    only to work ordered after them on that stream.  When the launch went to
    another stream, record that stream on them so that their memory is not
    reused before the launch has read them."""
    if stream is None or stream == torch.cuda.current_stream(tensors[0].device):
        return
    for t in tensors:
        t.record_stream(stream)


def _ptr_array(tensors, device):
    return torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64, device=device)


def lu_factor_batched(As, stream=None):
    """Factor a list of square CUDA matrices (all float64 or all float32,
    n <= 1024) in one launch, in place.  Returns (pivs, info) where pivs is
    a list of int32 CUDA tensors and info an int32 CUDA tensor (-1 marks an
    unsupported matrix)."""
    if not As:
        return [], None
    dt = As[0].dtype
    if dt not in (torch.float64, torch.float32):
        raise TypeError("batched matrices must be float64 or float32")
    dev = As[0].device
    for A in As:
        _require(A, "A", dt, 2)
        if A.shape[0] != A.shape[1]:
            raise ValueError("batched matrices must be square")
    pivs = [torch.empty(max(A.shape[0], 1), dtype=torch.int32, device=dev) for A in As]
    n = torch.tensor([A.shape[0] for A in As], dtype=torch.int32, device=dev)
    lda = torch.tensor([max(A.stride(0), 1) for A in As], dtype=torch.int32, device=dev)
    pa = _ptr_array(As, dev)
    pp = _ptr_array(pivs, dev)
    info = torch.empty(len(As), dtype=torch.int32, device=dev)
    prec = nat.LU_PREC_F64 if dt == torch.float64 else nat.LU_PREC_F32
    rc = nat.library().lu_factor_batched(len(As), n.data_ptr(), pa.data_ptr(), lda.data_ptr(), pp.data_ptr(),
                                         info.data_ptr(), prec, _stream_handle(stream))
    nat.check("lu_factor_batched", rc)
    _keep_for_stream(stream, n, lda, pa, pp)
    return [p[: A.shape[0]] for p, A in zip(pivs, As)], info


def lu_solve_batched(LUs, pivs, Bs, stream=None):
    """Solve each LU X = B in place (B: n x nrhs, nrhs <= 8), one launch."""
    if not LUs:
        return Bs
    dev = LUs[0].device
    dt = LUs[0].dtype
    Bs2 = [B if B.dim() == 2 else B.view(-1, 1) for B in Bs]
    n = torch.tensor([L.shape[0] for L in LUs], dtype=torch.int32, device=dev)
    nr = torch.tensor([B.shape[1] for B in Bs2], dtype=torch.int32, device=dev)
    lda = torch.tensor([max(L.stride(0), 1) for L in LUs], dtype=torch.int32, device=dev)
    ldb = torch.tensor([max(B.stride(0), 1) for B in Bs2], dtype=torch.int32, device=dev)
    pl, pp, pb = _ptr_array(LUs, dev), _ptr_array(pivs, dev), _ptr_array(Bs2, dev)
    prec = nat.LU_PREC_F64 if dt == torch.float64 else nat.LU_PREC_F32
    rc = nat.library().lu_solve_batched(len(LUs), n.data_ptr(), nr.data_ptr(), pl.data_ptr(), lda.data_ptr(),
                                        pp.data_ptr(), pb.data_ptr(), ldb.data_ptr(), prec, _stream_handle(stream))
    nat.check("lu_solve_batched", rc)
    _keep_for_stream(stream, n, nr, lda, ldb, pl, pp, pb)
    return Bs


def batched_panel_width(n: int, dtype=torch.float64) -> int:
    """Panel width b the batched factorization uses for an n x n matrix."""
    prec = nat.LU_PREC_F32 if dtype == torch.float32 else nat.LU_PREC_F64
    return int(nat.library().lu_batched_panel_width_dt(int(n), prec))


def set_batched_panel_widths(dtype, widths=None) -> None:
    """Replace the six size-class panel widths of the batched factorization
    for dtype (torch.float64 / float32); None restores the defaults."""
    prec = nat.LU_PREC_F32 if dtype == torch.float32 else nat.LU_PREC_F64
    if widths is None:
        nat.check("lu_batched_set_panel_widths", nat.library().lu_batched_set_panel_widths(prec, None, 6))
        return
    arr = (ctypes.c_int * len(widths))(*[int(w) for w in widths])
    nat.check("lu_batched_set_panel_widths", nat.library().lu_batched_set_panel_widths(prec, arr, len(widths)))


class BatchedFactorSolve:
    """lu_factor_batched followed by lu_solve_batched over fixed lists of
    matrices and right-hand sides, with the size and pointer arrays built
    once: restore() copies the inputs from the caller's pristine tensors into
    the work copies .A / .B, factor() and solve() are one C call each, and
    capture() records restore + factor + solve as one CUDA graph that
    replay() launches.  As / Bs are lists of CUDA tensors (float64 or
    float32, n <= 1024, nrhs <= 8) that stay owned by the caller.  Everything
    runs on self.stream."""

    def __init__(self, As, Bs):
        if not As or len(As) != len(Bs):
            raise ValueError("need matching, non-empty lists of matrices and right-hand sides")
        dt = As[0].dtype
        if dt not in (torch.float64, torch.float32):
            raise TypeError("batched matrices must be float64 or float32")
        dev = As[0].device
        self.A0, self.B0 = As, [B if B.dim() == 2 else B.view(-1, 1) for B in Bs]
        for A, B in zip(self.A0, self.B0):
            _require(A, "A", dt, 2)
            _require(B, "B", dt, 2)
        self.A = [a.clone() for a in self.A0]
        self.B = [b.clone() for b in self.B0]
        self.piv = [torch.empty(max(a.shape[0], 1), dtype=torch.int32, device=dev) for a in self.A]
        self.info = torch.empty(len(self.A), dtype=torch.int32, device=dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self._n = torch.tensor([a.shape[0] for a in self.A], **i32)
        self._lda = torch.tensor([max(a.stride(0), 1) for a in self.A], **i32)
        self._nr = torch.tensor([b.shape[1] for b in self.B], **i32)
        self._ldb = torch.tensor([max(b.stride(0), 1) for b in self.B], **i32)
        self._pa, self._pp, self._pb = _ptr_array(self.A, dev), _ptr_array(self.piv, dev), _ptr_array(self.B, dev)
        self._prec = nat.LU_PREC_F64 if dt == torch.float64 else nat.LU_PREC_F32
        self.stream = torch.cuda.Stream(device=dev)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        self.graph = None

    def restore(self):
        with torch.cuda.stream(self.stream):
            for a, a0 in zip(self.A, self.A0):
                a.copy_(a0)
            for b, b0 in zip(self.B, self.B0):
                b.copy_(b0)

    def factor(self):
        nat.check("lu_factor_batched", nat.library().lu_factor_batched(
            len(self.A), self._n.data_ptr(), self._pa.data_ptr(), self._lda.data_ptr(), self._pp.data_ptr(),
            self.info.data_ptr(), self._prec, ctypes.c_void_p(self.stream.cuda_stream)))

    def solve(self):
        nat.check("lu_solve_batched", nat.library().lu_solve_batched(
            len(self.A), self._n.data_ptr(), self._nr.data_ptr(), self._pa.data_ptr(), self._lda.data_ptr(),
            self._pp.data_ptr(), self._pb.data_ptr(), self._ldb.data_ptr(), self._prec,
            ctypes.c_void_p(self.stream.cuda_stream)))

    def capture(self):
        """Record restore + factor + solve as one CUDA graph (after one plain
        run, which sets kernel attributes and loads the device code)."""
        self.restore()
        self.factor()
        self.solve()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            self.restore()
            self.factor()
            self.solve()
        return self

    def replay(self):
        """One graph launch on self.stream (not synchronized)."""
        with torch.cuda.stream(self.stream):
            self.graph.replay()
