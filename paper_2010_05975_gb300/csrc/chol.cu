// Cholesky factorization A = L L^T (binary64 or binary32), no pivoting: the
// kernel Section 2.2 and the Conclusions name for the same schedule.  Blocked
// right-looking, like Algorithm 1 without TournPivot: per step k of width w,
//   1. L00 = chol(A00)                     (one CTA, this file)
//   2. L21 = A21 * L00^{-T}                (trsm_l21 with U = L00^T)
//   3. A22 -= L21 * L21^T, lower triangle  (syrk_lower)
// Every element receives its update terms fma(-l_ip, l_jp, a_ij) in
// ascending p and then its square root (diagonal) or one IEEE division, so
// the result is the column-by-column right-looking factorization bit for bit.
// Only the lower triangle is read or written.
#include "common.cuh"
#include "prof.cuh"

namespace lu {

// The w x w diagonal block, factored in shared memory (S, stride w + 1,
// lower triangle) one column at a time.  Writes L00 back to A and L00^T to
// Ut (w x w, row-major, upper triangle).  *info, if still 0, takes k + j + 1
// for the block's first column j whose pivot is not positive (or is NaN);
// the block is then finished anyway (sqrt of a negative is NaN, no trap).
template <typename T>
__global__ void __launch_bounds__(256) chol_diag_kernel(T* __restrict__ A, int lda, int k, int w, T* __restrict__ Ut,
                                                        int* __restrict__ info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    T* col = S + static_cast<size_t>(w) * (w + 1);     // column j of L below the diagonal
    __shared__ int s_bad;
    const int ws = w + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int i = warp; i < w; i += nwarp)
        for (int c = lane; c <= i; c += 32) S[i * ws + c] = A[idx(k + i, k + c, lda)];
    if (tid == 0) s_bad = -1;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            const T d = S[j * ws + j];
            if (!(d > T(0)) && s_bad < 0) s_bad = j;
            S[j * ws + j] = sqrt(d);
        }
        __syncthreads();
        const T ljj = S[j * ws + j];
        for (int i = j + 1 + tid; i < w; i += blockDim.x) {
            const T v = S[i * ws + j] / ljj;
            S[i * ws + j] = v;
            col[i] = v;
        }
        __syncthreads();
        // a_ic -= l_ij * l_cj for j < c <= i: warp rows, lane columns
        for (int i = j + 1 + warp; i < w; i += nwarp) {
            const T li = col[i];
            for (int c = j + 1 + lane; c <= i; c += 32) S[i * ws + c] = fma(-li, col[c], S[i * ws + c]);
        }
        __syncthreads();
    }
    for (int i = warp; i < w; i += nwarp)
        for (int c = lane; c <= i; c += 32) {
            const T v = S[i * ws + c];
            A[idx(k + i, k + c, lda)] = v;
            Ut[idx(c, i, w)] = v;
        }
    if (tid == 0 && s_bad >= 0 && *info == 0) *info = k + s_bad + 1;
}

template <typename T>
static int chol_diag(T* A, int lda, int k, int w, T* Ut, int* info, cudaStream_t s) {
    const size_t smem = (static_cast<size_t>(w) * (w + 1) + w) * sizeof(T);
    if (int rc = smem_attr(chol_diag_kernel<T>, smem)) return rc;
    {
        ProfScope ps(LU_PROF_CHOL_DIAG, s, static_cast<double>(w) * w * w / 3.0);
        chol_diag_kernel<T><<<1, 256, smem, s>>>(A, lda, k, w, Ut, info);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// Step loop with a one-panel lookahead (as the LU's): after step k's panel
// solve, the update of the NEXT panel's columns runs first; the next
// diagonal block and panel solve then run on a high-priority side stream
// beside the rest of the update, which does not touch those columns.
template <typename T>
static int chol_loop(int n, T* A, int lda, int* info, int b, cudaStream_t s) {
    LU_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    if (n == 0) return 0;
    T* Ut = nullptr;
    if (lu_malloc_async(reinterpret_cast<void**>(&Ut), static_cast<size_t>(b) * b * sizeof(T), s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    int lo = 0, hi = 0, rc = 0;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_next = nullptr;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_next, cudaEventDisableTiming) != cudaSuccess)
        rc = LU_ELAUNCH;
    {
        const int w0 = n < b ? n : b;
        if (!rc) rc = chol_diag<T>(A, lda, 0, w0, Ut, info, s);
        if (!rc) rc = trsm_l21<T>(A, lda, n, 0, w0, Ut, w0, s);
    }
    for (int k = 0; k < n && rc == 0; k += b) {
        const int w = (n - k) < b ? (n - k) : b;
        const int kn = k + w;
        const int wn = (n - kn) < b ? (n - kn) : b;     // next panel width (<= 0: none)
        if (wn <= 0) break;
        rc = syrk_lower<T>(A, lda, n, k, w, kn, kn + wn, s);
        if (!rc && cudaEventRecord(ev_panel, s) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc && cudaStreamWaitEvent(s2, ev_panel, 0) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = chol_diag<T>(A, lda, kn, wn, Ut, info, s2);
        if (!rc) rc = trsm_l21<T>(A, lda, n, kn, wn, Ut, wn, s2);
        if (!rc && cudaEventRecord(ev_next, s2) != cudaSuccess) rc = LU_ELAUNCH;
        if (!rc) rc = syrk_lower<T>(A, lda, n, k, w, kn + wn, n, s);
        if (!rc && cudaStreamWaitEvent(s, ev_next, 0) != cudaSuccess) rc = LU_ELAUNCH;
    }
    // join the side stream before the workspace goes back to the pool
    if (s2 && ev_next) {
        cudaEventRecord(ev_next, s2);
        cudaStreamWaitEvent(s, ev_next, 0);
    }
    cudaFreeAsync(Ut, s);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_next) cudaEventDestroy(ev_next);
    if (s2) cudaStreamDestroy(s2);
    return rc;
}

static int chol_args(int n, const void* A, int lda, const int* info, const lu_opts* opts, int elem, int& b) {
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (info == nullptr) return -4;
    b = (n >= 4096) ? 128 : 64;
    if (opts) {
        if (opts->b < 0 || opts->h != 0 || opts->defer != 0) return -5;
        if (opts->precision != (elem == 8 ? LU_PREC_F64 : LU_PREC_F32) && opts->precision != 0) return -5;
        for (int r : opts->reserved)
            if (r != 0) return -5;
        if (opts->b > 0) b = opts->b;
    }
    if (b > kCholMaxPanel) return -5;
    return 0;
}

}  // namespace lu

using namespace lu;

extern "C" int chol_factor(int n, double* A, int lda, int* info, const lu_opts* opts, cudaStream_t stream) {
    int b;
    if (int rc = chol_args(n, A, lda, info, opts, 8, b)) return rc;
    return chol_loop<double>(n, A, lda, info, b, stream);
}

extern "C" int chol_factor_f32(int n, float* A, int lda, int* info, const lu_opts* opts, cudaStream_t stream) {
    int b;
    if (int rc = chol_args(n, A, lda, info, opts, 4, b)) return rc;
    return chol_loop<float>(n, A, lda, info, b, stream);
}
