// C ABI: argument validation and the step loop of the blocked factorization
// (Algorithm 1 on one GPU: TournPivot -> apply pivots -> FactorizeA10 ->
// FactorizeA01 -> FactorizeA11, then the active block shrinks by w).
#include "common.cuh"

namespace lu {

// The library's memory pools, one per device (see lu_malloc_async).
static cudaError_t lib_pool(cudaMemPool_t* out) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = pools.find(dev);
        if (it != pools.end()) {
            pool = it->second;
        } else {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaError_t e = cudaMemPoolCreate(&pool, &props)) return e;
            unsigned long long keep = 16ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = pool;
        }
    }
    *out = pool;
    return cudaSuccess;
}

cudaError_t lu_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    if (cudaError_t e = lib_pool(&pool)) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}


struct FactorWs {
    int* lists = nullptr;
    int* counts = nullptr;
    void* a00 = nullptr;
    int* mv = nullptr;
    size_t stride_nodes = 0;
};

static void ws_free(FactorWs& ws, cudaStream_t s) {
    if (ws.lists) cudaFreeAsync(ws.lists, s);
    if (ws.counts) cudaFreeAsync(ws.counts, s);
    if (ws.a00) cudaFreeAsync(ws.a00, s);
    if (ws.mv) cudaFreeAsync(ws.mv, s);
    ws = FactorWs{};
}

static int ws_alloc(FactorWs& ws, int m, int b, int h, size_t elem, cudaStream_t s) {
    ws.stride_nodes = static_cast<size_t>(cdiv(m, h > 0 ? h : 1)) + 1;
    bool ok = lu_malloc_async(reinterpret_cast<void**>(&ws.lists), 2 * ws.stride_nodes * b * sizeof(int), s) == cudaSuccess &&
              lu_malloc_async(reinterpret_cast<void**>(&ws.counts), 4 * ws.stride_nodes * sizeof(int), s) == cudaSuccess &&
              lu_malloc_async(&ws.a00, static_cast<size_t>(b) * b * elem, s) == cudaSuccess &&
              lu_malloc_async(reinterpret_cast<void**>(&ws.mv), (1 + 4 * static_cast<size_t>(b)) * sizeof(int), s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ws_free(ws, s);
        return LU_ENOMEM;
    }
    return 0;
}

static bool tslu_shapes_fit(int m, int kmax, int b, int h, int elem) {
    for (int k = 0; k < kmax; k += b) {
        const int w = (kmax - k) < b ? (kmax - k) : b;
        if (tslu_shape(m, k, w, h, kTsluMaxCluster, elem).smem > kTsluSmemLimit) return false;
    }
    return true;
}

// Schur update of columns [c0, c1) for one step, by arithmetic.
struct SchurF64 {
    int operator()(double* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s) const {
        return schur_f64(A, lda, m, k, w, c0, c1, s);
    }
};
struct SchurF32 {
    int operator()(float* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s) const {
        return schur_f32(A, lda, m, k, w, c0, c1, s);
    }
};

// Step loop with a one-panel lookahead.  On the caller's stream s, step t
// runs: wait for its tournament -> apply pivots -> L21, U12 -> the Schur
// update of the NEXT panel's columns -> (fork) the rest of the Schur update.
// The next tournament reads only those panel columns, so it runs on a
// high-priority side stream concurrently with the rest of the update; the
// next step's pivot application waits for both.
struct NoRowsDone {
    int operator()(int, int, cudaEvent_t) const { return 0; }
};

// `done(k, kn, ready)` runs once step k has enqueued all its work: rows
// [k, kn) are then final in every column once `ready` has fired (later steps
// swap and update only rows >= kn).
template <typename T, typename Schur, typename RowsDone = NoRowsDone>
static int factor_loop(int m, int n, T* A, int lda, int* piv, int* info, int b, int h, const Schur& schur,
                       cudaStream_t s, const RowsDone& done = RowsDone{}) {
    LU_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    const int kmax = m < n ? m : n;
    if (kmax == 0) return 0;
    FactorWs ws;
    if (int rc = ws_alloc(ws, m, b, h, sizeof(T), s)) return rc;
    T* a00 = static_cast<T*>(ws.a00);
    int lo = 0, hi = 0;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_tslu = nullptr, ev_piv = nullptr, ev_u12 = nullptr;
    int rc = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_tslu, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_piv, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_u12, cudaEventDisableTiming) != cudaSuccess)
        rc = LU_ELAUNCH;
    const int* root = nullptr;
    if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc) rc = tslu_select<T>(A, lda, m, 0, (kmax < b ? kmax : b), h, ws.lists, ws.counts, ws.stride_nodes, a00,
                                 info, &root, s2);
    if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
    for (int k = 0; k < kmax && rc == 0; k += b) {
        const int w = (kmax - k) < b ? (kmax - k) : b;
        const int kn = k + w;
        const int wn = (kmax - kn) < b ? (kmax - kn) : b;     // next panel width (<= 0: none)
        if (cudaStreamWaitEvent(s, ev_tslu, 0) != cudaSuccess) { rc = LU_ELAUNCH; break; }
        rc = pivot_apply<T>(A, lda, m, n, k, w, root, a00, piv, ws.mv, s);
        // L21 (rows below the panel) and U12 (columns right of it) only read
        // A00: U12 runs on the side stream beside L21, filling each other's
        // last waves.
        if (!rc && cudaEventRecord(ev_piv, s) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc && cudaStreamWaitEvent(s2, ev_piv, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = trsm_u12<T>(A, lda, n, k, w, s2);
        if (!rc && cudaEventRecord(ev_u12, s2) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = trsm_l21<T>(A, lda, m, k, w, A + idx(k, k, lda), lda, s);
        if (!rc && cudaStreamWaitEvent(s, ev_u12, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (rc) break;
        if (wn > 0) {
            rc = schur(A, lda, m, k, w, kn, kn + wn, s);
            if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc) rc = tslu_select<T>(A, lda, m, kn, wn, h, ws.lists, ws.counts, ws.stride_nodes, a00, info,
                                         &root, s2);
            if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc) rc = schur(A, lda, m, k, w, kn + wn, n, s);
        } else {
            rc = schur(A, lda, m, k, w, kn, n, s);
        }
        // ev_u12 follows this step's row moves (through ev_piv) and its U12
        if (!rc) rc = done(k, kn, ev_u12);
    }
    // join the side stream before the workspace goes back to the pool
    if (ev_tslu && s2) {
        cudaEventRecord(ev_tslu, s2);
        cudaStreamWaitEvent(s, ev_tslu, 0);
    }
    ws_free(ws, s);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_tslu) cudaEventDestroy(ev_tslu);
    if (ev_piv) cudaEventDestroy(ev_piv);
    if (ev_u12) cudaEventDestroy(ev_u12);
    if (s2) cudaStreamDestroy(s2);
    return rc;
}

// Shared argument checks of the factor entry points.  Returns 0 and fills
// b, h, prec, or a negative argument index.
static int factor_args(int m, int n, const void* A, int lda, const int* piv, const int* info, const lu_opts* opts,
                       int elem, int& b, int& h, int& prec, int* defer = nullptr) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    const int kmax = m < n ? m : n;
    if (kmax > 0 && A == nullptr) return -3;
    if (kmax > 0 && piv == nullptr) return -5;
    if (info == nullptr) return -6;
    b = (n >= 4096) ? 256 : 32;
    h = 128;
    prec = (elem == 8) ? LU_PREC_F64 : LU_PREC_F32;
    if (defer) *defer = 0;
    if (opts) {
        if (opts->b < 0 || opts->h < 0) return -7;
        if (opts->defer < 0 || opts->defer > kTcMaxPanels) return -7;
        if (defer) *defer = opts->defer;
        for (int r : opts->reserved)
            if (r != 0) return -7;
        if (opts->b > 0) b = opts->b;
        if (opts->h > 0) h = opts->h;
        if (opts->precision != 0 || elem == 8) prec = opts->precision;
    }
    if (b > kMaxPanel) return -7;
    if (kmax > 0 && !tslu_shapes_fit(m, kmax, b, h, elem)) return -7;
    return 0;
}

// The bf16 / fp8 factorization with deferred trailing updates (the reuse
// of Section 4.1 and the per-step update cost of Section 7.4 applied to HBM:
// each pass over the trailing matrix applies up to `defer` panels).  Each
// step quantizes its L21 and U12 once and adds them to the pending list.
// Elements receive the pending panels in step order, each as
// C = fma(-s_p, acc_p, C) with acc_p one panel's fp32 product, so the factors
// are those of one full trailing update per step, bit for bit:
//   - after the step's row swaps, the rows of every pending Lq (and their
//     fp8 exponents) make the same moves, so each row keeps its operands;
//   - the winners' rows right of the panel (the "row strip") receive the
//     pending panels before the U12 solve reads them;
//   - the next panel's columns (the "column strip") receive all pending
//     panels before the next tournament reads them;
//   - the rest of the trailing matrix receives them in one pass when
//     `defer` panels are pending.
static int factor_lowp(int m, int n, float* A, int lda, int* piv, int* info, int b, int h, int prec, int defer,
                       cudaStream_t s) {
    if (m != n || (b % 128) != 0) return LU_EUNSUPPORTED;
    LU_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    const int kmax = n;
    if (kmax == 0) return 0;
    const bool fp8 = prec == LU_PREC_FP8;
    const size_t elem = fp8 ? 1 : 2;
    const int d = defer > 0 ? defer : kDeferDefault;
    struct Slot {
        unsigned char* Lq = nullptr;
        unsigned char* Uq = nullptr;
        int* eLrow = nullptr;
        int* eU = nullptr;
    } slot[kTcMaxPanels];
    const size_t nblk = static_cast<size_t>(cdiv(n, 256)) + 1;
    bool ok = true;
    for (int i = 0; i < d && ok; ++i)
        ok = lu_malloc_async(reinterpret_cast<void**>(&slot[i].Lq), static_cast<size_t>(m) * kLowpK * elem + 256, s) == cudaSuccess &&
             lu_malloc_async(reinterpret_cast<void**>(&slot[i].Uq), static_cast<size_t>(n) * kLowpK * elem + 256, s) == cudaSuccess &&
             lu_malloc_async(reinterpret_cast<void**>(&slot[i].eLrow), (static_cast<size_t>(m) + 1) * sizeof(int), s) == cudaSuccess &&
             lu_malloc_async(reinterpret_cast<void**>(&slot[i].eU), nblk * sizeof(int), s) == cudaSuccess;
    FactorWs ws;
    int rc = ok ? ws_alloc(ws, m, b, h, sizeof(float), s) : LU_ENOMEM;
    float* a00 = static_cast<float*>(ws.a00);
    int lo = 0, hi = 0;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_tslu = nullptr, ev_piv = nullptr, ev_u12 = nullptr;
    if (!rc && (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
                cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_tslu, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_piv, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_u12, cudaEventDisableTiming) != cudaSuccess))
        rc = LU_ELAUNCH;
    LowpOperand P[kTcMaxPanels];
    int np = 0;
    const int* root = nullptr;
    if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc) rc = tslu_select<float>(A, lda, m, 0, (kmax < b ? kmax : b), h, ws.lists, ws.counts, ws.stride_nodes, a00,
                                     info, &root, s2);
    if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
    for (int k = 0; k < kmax && rc == 0; k += b) {
        const int w = (kmax - k) < b ? (kmax - k) : b;
        const int kn = k + w;
        const int wn = (kmax - kn) < b ? (kmax - kn) : b;     // next panel width (<= 0: none)
        if (cudaStreamWaitEvent(s, ev_tslu, 0) != cudaSuccess) { rc = LU_ELAUNCH; break; }
        rc = pivot_apply<float>(A, lda, m, n, k, w, root, a00, piv, ws.mv, s);
        if (!rc && np > 0) rc = lowp_row_moves(P, np, fp8, ws.mv, w, s);
        // the winners' rows right of the panel receive the pending panels
        if (!rc && np > 0) rc = schur_tc_apply(A, lda, k, kn, w, n - kn, P, np, fp8, info, false, s);
        if (!rc && cudaEventRecord(ev_piv, s) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc && cudaStreamWaitEvent(s2, ev_piv, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = trsm_u12<float>(A, lda, n, k, w, s2);
        if (!rc && cudaEventRecord(ev_u12, s2) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = trsm_l21<float>(A, lda, m, k, w, A + idx(k, k, lda), lda, s);
        if (!rc && cudaStreamWaitEvent(s, ev_u12, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (rc || kn >= n) break;
        // this step's operands join the pending list
        Slot& sl = slot[np];
        rc = quantize_l21(A, lda, m, k, w, fp8, sl.Lq, sl.eLrow, s);
        if (!rc) rc = quantize_u12(A, lda, k, w, kn, n, fp8, sl.Uq, sl.eU, s);
        if (rc) break;
        P[np++] = LowpOperand{sl.Lq, m - kn, sl.eLrow, sl.Uq, n - kn, sl.eU, kn, kn, w};
        // the next panel's columns, then its tournament beside the rest
        rc = schur_tc_apply(A, lda, kn, kn, m - kn, wn, P, np, fp8, info, false, s);
        if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = tslu_select<float>(A, lda, m, kn, wn, h, ws.lists, ws.counts, ws.stride_nodes, a00, info,
                                         &root, s2);
        if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc && np == d) {
            rc = schur_tc_apply(A, lda, kn, kn + wn, m - kn, n - kn - wn, P, np, fp8, info, true, s);
            np = 0;
        }
    }
    // join the side stream before the workspace goes back to the pool
    if (ev_tslu && s2) {
        cudaEventRecord(ev_tslu, s2);
        cudaStreamWaitEvent(s, ev_tslu, 0);
    }
    cudaGetLastError();
    ws_free(ws, s);
    for (int i = 0; i < kTcMaxPanels; ++i) {
        if (slot[i].Lq) cudaFreeAsync(slot[i].Lq, s);
        if (slot[i].Uq) cudaFreeAsync(slot[i].Uq, s);
        if (slot[i].eLrow) cudaFreeAsync(slot[i].eLrow, s);
        if (slot[i].eU) cudaFreeAsync(slot[i].eU, s);
    }
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_tslu) cudaEventDestroy(ev_tslu);
    if (ev_piv) cudaEventDestroy(ev_piv);
    if (ev_u12) cudaEventDestroy(ev_u12);
    if (s2) cudaStreamDestroy(s2);
    return rc;
}

}  // namespace lu

using namespace lu;

extern "C" int lu_gemm_lowp(int M, int N, int K, const float* L, int ldl, const float* U, int ldu, float* C, int ldc,
                            int precision, int* status, cudaStream_t stream) {
    if (M < 0) return -1;
    if (N < 0) return -2;
    if (K < 0 || K > kLowpK) return -3;
    if (M > 0 && K > 0 && (L == nullptr || ldl < K)) return -4;
    if (N > 0 && K > 0 && (U == nullptr || ldu < N)) return -6;
    if (M > 0 && N > 0 && (C == nullptr || ldc < N)) return -8;
    if (precision != LU_PREC_BF16 && precision != LU_PREC_FP8) return -10;
    if (status == nullptr) return -11;
    LU_TRY(cudaMemsetAsync(status, 0, sizeof(int), stream));
    if (M == 0 || N == 0 || K == 0) return 0;
    const bool fp8 = precision == LU_PREC_FP8;
    const size_t elem = fp8 ? 1 : 2;
    unsigned char *Lq = nullptr, *Uq = nullptr;
    int *eL = nullptr, *eU = nullptr;
    bool ok = lu_malloc_async(reinterpret_cast<void**>(&Lq), static_cast<size_t>(M) * kLowpK * elem + 256, stream) == cudaSuccess &&
              lu_malloc_async(reinterpret_cast<void**>(&Uq), static_cast<size_t>(N) * kLowpK * elem + 256, stream) == cudaSuccess &&
              lu_malloc_async(reinterpret_cast<void**>(&eL), (static_cast<size_t>(M) + 1) * sizeof(int), stream) == cudaSuccess &&
              lu_malloc_async(reinterpret_cast<void**>(&eU), (static_cast<size_t>(cdiv(N, 256)) + 1) * sizeof(int), stream) == cudaSuccess;
    int rc = LU_ENOMEM;
    if (ok) {
        // The quantizers read the operands as blocks of one matrix: L as
        // rows [r0, r0+M) x columns [k, k+K) and U as rows [k, k+K) x columns
        // [c0, c0+N).  Offsetting the base pointers maps L and U there with
        // k = 0, r0 = K for L and c0 = K for U.
        rc = quantize_l21(L - static_cast<ptrdiff_t>(K) * ldl, ldl, K + M, 0, K, fp8, Lq, eL, stream);
        if (!rc) rc = quantize_u12(U - K, ldu, 0, K, K, K + N, fp8, Uq, eU, stream);
        const LowpOperand op{Lq, M, eL, Uq, N, eU, 0, 0, K};
        if (!rc) rc = schur_tc_apply(C, ldc, 0, 0, M, N, &op, 1, fp8, status, false, stream);
    }
    cudaGetLastError();
    if (Lq) cudaFreeAsync(Lq, stream);
    if (Uq) cudaFreeAsync(Uq, stream);
    if (eL) cudaFreeAsync(eL, stream);
    if (eU) cudaFreeAsync(eU, stream);
    return rc;
}

extern "C" int lu_factor_ex(int m, int n, double* A, int lda, int* piv, int* info, const lu_opts* opts,
                            cudaStream_t stream) {
    int b, h, prec;
    if (int rc = factor_args(m, n, A, lda, piv, info, opts, 8, b, h, prec)) return rc;
    if (prec != LU_PREC_F64) return LU_EUNSUPPORTED;
    return factor_loop<double>(m, n, A, lda, piv, info, b, h, SchurF64{}, stream);
}

extern "C" int lu_memory_pool(void** pool) {
    if (pool == nullptr) return -1;
    cudaMemPool_t p = nullptr;
    if (lib_pool(&p) != cudaSuccess) {
        cudaGetLastError();
        return LU_ELAUNCH;
    }
    *pool = static_cast<void*>(p);
    return 0;
}

extern "C" int lu_factor_host(int m, int n, double* A, int lda, int* piv, int* info, const lu_opts* opts,
                              cudaStream_t stream) {
    int b, h, prec;
    if (int rc = factor_args(m, n, A, lda, piv, info, opts, 8, b, h, prec)) return rc;
    if (prec != LU_PREC_F64) return LU_EUNSUPPORTED;
    const int kmax = m < n ? m : n;
    *info = 0;
    if (kmax == 0) return 0;
    const size_t row = static_cast<size_t>(n) * sizeof(double);
    double* dA = nullptr;
    int* dpiv = nullptr;
    if (lu_malloc_async(reinterpret_cast<void**>(&dA), row * m, stream) != cudaSuccess ||
        lu_malloc_async(reinterpret_cast<void**>(&dpiv), (static_cast<size_t>(kmax) + 1) * sizeof(int), stream) !=
            cudaSuccess) {
        cudaGetLastError();
        if (dA) cudaFreeAsync(dA, stream);
        return LU_ENOMEM;
    }
    int* dinfo = dpiv + kmax;
    int rc = 0;
    // a contiguous matrix moves as one linear copy each way (a pitched copy
    // of 8.6 GB may be split into row transfers)
    const bool contig = (lda == n);
    const size_t hpitch = static_cast<size_t>(lda) * sizeof(double);
    // rows [r0, r1) of the device copy back to A on stream cs
    auto rows_back = [&](int r0, int r1, cudaStream_t cs) {
        if (r1 <= r0) return cudaSuccess;
        const double* src = dA + static_cast<size_t>(r0) * n;
        double* dst = A + static_cast<size_t>(r0) * lda;
        const size_t nr = static_cast<size_t>(r1 - r0);
        return contig ? cudaMemcpyAsync(dst, src, row * nr, cudaMemcpyDeviceToHost, cs)
                      : cudaMemcpy2DAsync(dst, hpitch, src, row, row, nr, cudaMemcpyDeviceToHost, cs);
    };
    if ((contig ? cudaMemcpyAsync(dA, A, row * static_cast<size_t>(m), cudaMemcpyHostToDevice, stream)
                : cudaMemcpy2DAsync(dA, row, A, hpitch, row, m, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        rc = LU_ELAUNCH;
    // With page-locked host memory each step's finished rows go back on a
    // copy stream while later steps run (a copy into pageable memory would
    // block this thread until the step finished, so those rows go back at
    // the end).  The copies then use the link throughout the factorization
    // instead of as one 8.6 GB transfer after it.
    cudaPointerAttributes attr{};
    const bool pinned = cudaPointerGetAttributes(&attr, A) == cudaSuccess && attr.type == cudaMemoryTypeHost;
    cudaGetLastError();
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_cs = nullptr;
    if (pinned && (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
                   cudaEventCreateWithFlags(&ev_cs, cudaEventDisableTiming) != cudaSuccess))
        rc = LU_ELAUNCH;
    int sent = 0;  // rows [0, sent) are on their way back
    auto done = [&](int k, int kn, cudaEvent_t ready) {
        if (!cs) return 0;
        if (cudaStreamWaitEvent(cs, ready, 0) != cudaSuccess || rows_back(k, kn, cs) != cudaSuccess)
            return static_cast<int>(LU_ELAUNCH);
        sent = kn;
        return 0;
    };
    if (!rc) rc = factor_loop<double>(m, n, dA, n, dpiv, dinfo, b, h, SchurF64{}, stream, done);
    if (!rc && (rows_back(sent, m, stream) != cudaSuccess ||
                cudaMemcpyAsync(piv, dpiv, static_cast<size_t>(kmax) * sizeof(int), cudaMemcpyDeviceToHost,
                                stream) != cudaSuccess ||
                cudaMemcpyAsync(info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess))
        rc = LU_ELAUNCH;
    // the copy stream reads dA: join it before dA goes back to the pool
    if (cs) {
        if (ev_cs) {
            cudaEventRecord(ev_cs, cs);
            cudaStreamWaitEvent(stream, ev_cs, 0);
        } else {
            cudaStreamSynchronize(cs);
        }
    }
    cudaGetLastError();
    cudaFreeAsync(dA, stream);
    cudaFreeAsync(dpiv, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess && !rc) rc = LU_ELAUNCH;
    if (ev_cs) cudaEventDestroy(ev_cs);
    if (cs) cudaStreamDestroy(cs);
    return rc;
}

extern "C" int lu_factor_f32(int m, int n, float* A, int lda, int* piv, int* info, const lu_opts* opts,
                             cudaStream_t stream) {
    int b, h, prec, defer;
    if (int rc = factor_args(m, n, A, lda, piv, info, opts, 4, b, h, prec, &defer)) return rc;
    if (prec == LU_PREC_F32) return factor_loop<float>(m, n, A, lda, piv, info, b, h, SchurF32{}, stream);
    if (prec == LU_PREC_BF16 || prec == LU_PREC_FP8)
        return factor_lowp(m, n, A, lda, piv, info, b, h, prec, defer, stream);
    return -7;
}

extern "C" int lu_factor(int n, double* A, int lda, int* piv, int* info, cudaStream_t stream) {
    if (n < 0) return -1;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (n > 0 && A == nullptr) return -2;
    if (n > 0 && piv == nullptr) return -4;
    if (info == nullptr) return -5;
    return lu_factor_ex(n, n, A, lda, piv, info, nullptr, stream);
}

extern "C" int lu_solve(int n, int nrhs, const double* LU, int lda, const int* piv, double* B, int ldb,
                        cudaStream_t stream) {
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > 384) return -2;
    if (n > 0 && LU == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && piv == nullptr) return -5;
    if (n > 0 && nrhs > 0 && B == nullptr) return -6;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -7;
    return getrs_f64(n, nrhs, LU, lda, piv, B, ldb, stream);
}

extern "C" int lu_solve_f32(int n, int nrhs, const float* LU, int lda, const int* piv, float* B, int ldb,
                            cudaStream_t stream) {
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > 384) return -2;
    if (n > 0 && LU == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && piv == nullptr) return -5;
    if (n > 0 && nrhs > 0 && B == nullptr) return -6;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -7;
    return getrs_f32(n, nrhs, LU, lda, piv, B, ldb, stream);
}
