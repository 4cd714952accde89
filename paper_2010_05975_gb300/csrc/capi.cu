// C ABI: argument validation and the step loop of the blocked factorization
// (Algorithm 1 on one GPU: TournPivot -> apply pivots -> FactorizeA10 ->
// FactorizeA01 -> FactorizeA11, then the active block shrinks by w).
#include "common.cuh"

namespace lu {

struct FactorWs {
    int* lists = nullptr;
    int* counts = nullptr;
    double* a00 = nullptr;
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

static int ws_alloc(FactorWs& ws, int m, int b, int h, cudaStream_t s) {
    ws.stride_nodes = static_cast<size_t>(cdiv(m, h > 0 ? h : 1)) + 1;
    bool ok = cudaMallocAsync(reinterpret_cast<void**>(&ws.lists), 2 * ws.stride_nodes * b * sizeof(int), s) == cudaSuccess &&
              cudaMallocAsync(reinterpret_cast<void**>(&ws.counts), 2 * ws.stride_nodes * sizeof(int), s) == cudaSuccess &&
              cudaMallocAsync(reinterpret_cast<void**>(&ws.a00), static_cast<size_t>(b) * b * sizeof(double), s) == cudaSuccess &&
              cudaMallocAsync(reinterpret_cast<void**>(&ws.mv), (1 + 4 * static_cast<size_t>(b)) * sizeof(int), s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ws_free(ws, s);
        return LU_ENOMEM;
    }
    return 0;
}

// Largest dynamic shared memory a tournament CTA may take (the kernel also
// uses ~1 KB of static shared memory).
constexpr size_t kTsluSmemLimit = 232448 - 2048;

static bool tslu_shapes_fit(int m, int kmax, int b, int h) {
    for (int k = 0; k < kmax; k += b) {
        const int w = (kmax - k) < b ? (kmax - k) : b;
        if (tslu_shape(m, k, w, h, kTsluMaxCluster).smem > kTsluSmemLimit) return false;
    }
    return true;
}

// Step loop with a one-panel lookahead.  On the caller's stream s, step t
// runs: wait for its tournament -> apply pivots -> L21, U12 -> the Schur
// update of the NEXT panel's columns -> (fork) the rest of the Schur update.
// The next tournament reads only those panel columns, so it runs on a
// high-priority side stream concurrently with the rest of the update; the
// next step's pivot application waits for both.
static int factor_f64(int m, int n, double* A, int lda, int* piv, int* info, int b, int h, cudaStream_t s) {
    LU_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    const int kmax = m < n ? m : n;
    if (kmax == 0) return 0;
    FactorWs ws;
    if (int rc = ws_alloc(ws, m, b, h, s)) return rc;
    int lo = 0, hi = 0;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_tslu = nullptr;
    int rc = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_tslu, cudaEventDisableTiming) != cudaSuccess)
        rc = LU_ELAUNCH;
    const int* root = nullptr;
    if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc) rc = tslu_select_f64(A, lda, m, 0, (kmax < b ? kmax : b), h, ws.lists, ws.counts, ws.stride_nodes,
                                  ws.a00, info, &root, s2);
    if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
    for (int k = 0; k < kmax && rc == 0; k += b) {
        const int w = (kmax - k) < b ? (kmax - k) : b;
        const int kn = k + w;
        const int wn = (kmax - kn) < b ? (kmax - kn) : b;     // next panel width (<= 0: none)
        if (cudaStreamWaitEvent(s, ev_tslu, 0) != cudaSuccess) { rc = LU_ELAUNCH; break; }
        rc = pivot_apply_f64(A, lda, m, n, k, w, root, ws.a00, piv, ws.mv, s);
        if (!rc) rc = trsm_l21_f64(A, lda, m, k, w, s);
        if (!rc) rc = trsm_u12_f64(A, lda, n, k, w, s);
        if (rc) break;
        if (wn > 0) {
            rc = schur_f64(A, lda, m, k, w, kn, kn + wn, s);
            if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc) rc = tslu_select_f64(A, lda, m, kn, wn, h, ws.lists, ws.counts, ws.stride_nodes, ws.a00,
                                          info, &root, s2);
            if (!rc && cudaEventRecord(ev_tslu, s2) != cudaSuccess) rc = LU_ELAUNCH;
            if (!rc) rc = schur_f64(A, lda, m, k, w, kn + wn, n, s);
        } else {
            rc = schur_f64(A, lda, m, k, w, kn, n, s);
        }
    }
    // join the side stream before the workspace goes back to the pool
    if (ev_tslu && s2) {
        cudaEventRecord(ev_tslu, s2);
        cudaStreamWaitEvent(s, ev_tslu, 0);
    }
    ws_free(ws, s);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_tslu) cudaEventDestroy(ev_tslu);
    if (s2) cudaStreamDestroy(s2);
    return rc;
}

}  // namespace lu

using namespace lu;

extern "C" int lu_factor_ex(int m, int n, double* A, int lda, int* piv, int* info, const lu_opts* opts,
                            cudaStream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    const int kmax = m < n ? m : n;
    if (kmax > 0 && A == nullptr) return -3;
    if (kmax > 0 && piv == nullptr) return -5;
    if (info == nullptr) return -6;
    int b = (n >= 4096) ? 256 : 32, h = 128, prec = LU_PREC_F64;
    if (opts) {
        if (opts->b < 0 || opts->h < 0) return -7;
        for (int r : opts->reserved)
            if (r != 0) return -7;
        if (opts->b > 0) b = opts->b;
        if (opts->h > 0) h = opts->h;
        prec = opts->precision;
    }
    if (b > kMaxPanel) return -7;
    if (prec != LU_PREC_F64) return LU_EUNSUPPORTED;
    if (kmax > 0 && !tslu_shapes_fit(m, kmax, b, h)) return -7;
    return factor_f64(m, n, A, lda, piv, info, b, h, stream);
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
