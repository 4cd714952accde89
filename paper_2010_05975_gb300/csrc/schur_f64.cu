// FactorizeA11 (Section 7.2) in binary64: A22 -= L21 * U12, K = w <= 256.
//
// GB300 executes binary64 on the CUDA cores only (no tcgen05 kind for it;
// measured DFMA ~1.19 TFLOP/s per GPU, DMMA m8n8k4 slower), so this is a
// register-tiled DFMA kernel: a CTA tile of BM x BN outputs, 256 threads,
// TM x TN accumulators per thread, K staged through shared memory in
// double-buffered chunks of 8.  Each accumulator starts from the A22 value
// and receives fma(-l, u, acc) for p = 0, 1, ..., w-1, the oracle's order, so
// the result is bit-identical to it.
//
// The same kernel, instantiated with SYRK, is the symmetric update of the
// Cholesky factorization: the lower triangle (r >= c) of rows [c0, m) x
// columns [c0, c1) receives -= L21 * L21^T, both operands read from the rows
// of L21 (columns [k, k+w)).  TRI enumerates only the tiles of the square's
// lower triangle (c1 = m); without it the grid is a rectangle (a panel of
// columns) and tiles wholly above the diagonal exit at once.
#include "common.cuh"
#include "prof.cuh"

namespace lu {

template <typename T, int BM, int BN, bool SYRK = false, bool TRI = false>
__global__ void __launch_bounds__(256) schur_simt_kernel(T* __restrict__ A, int lda, int m, int k, int w, int c0,
                                                         int n) {
    static_assert(!SYRK || BM == BN, "the symmetric update uses square tiles");
    constexpr int BK = 8;
    constexpr int TM = BM / 16, TN = BN / 16;
    constexpr int APT = BM * BK / 256;          // A elements loaded per thread per chunk
    constexpr int BPT = BN * BK / 256;          // B elements loaded per thread per chunk
    constexpr int BTPR = BN / BPT;              // threads per B row
    __shared__ T As[2][BK][BM];
    __shared__ T Bs[2][BK][BN];

    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    int row0, col0;
    if (SYRK && TRI) {
        // tile t = ti (ti + 1) / 2 + tj of the lower triangle, tj <= ti
        const long long t = blockIdx.x;
        long long ti = static_cast<long long>((sqrt(8.0 * static_cast<double>(t) + 1.0) - 1.0) * 0.5);
        while (ti * (ti + 1) / 2 > t) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        const long long tj = t - ti * (ti + 1) / 2;
        row0 = c0 + static_cast<int>(ti) * BM;
        col0 = c0 + static_cast<int>(tj) * BN;
    } else {
        row0 = (SYRK ? c0 : k + w) + blockIdx.y * BM;
        col0 = c0 + blockIdx.x * BN;
    }
    if (SYRK && col0 > row0 + BM - 1) return;   // wholly above the diagonal

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            acc[i][j] = (r < m && c < n && (!SYRK || r >= c)) ? A[idx(r, c, lda)] : T(0);
        }

    // loader coordinates (SYRK: B^T is read like A, from the rows col0 + b_r)
    const int a_r = tid % BM, a_k = (tid / BM) * APT;
    const int b_k = SYRK ? (tid / BN) * BPT : tid / BTPR;
    const int b_c = SYRK ? tid % BN : (tid % BTPR) * BPT;
    const bool a_row_ok = (row0 + a_r) < m;
    const bool b_row_ok = (col0 + b_c) < n;
    const T* a_src = A + idx(row0 + a_r < m ? row0 + a_r : row0, k, lda);
    const T* b_src = SYRK ? A + idx(b_row_ok ? col0 + b_c : col0, k, lda) : A + idx(k, col0 + b_c, lda);

    T ra[APT], rb[BPT];
    auto load_chunk = [&](int kc) {
#pragma unroll
        for (int e = 0; e < APT; ++e) {
            const int kk = kc + a_k + e;
            ra[e] = (a_row_ok && kk < w) ? a_src[kk] : T(0);
        }
        if (SYRK) {
#pragma unroll
            for (int e = 0; e < BPT; ++e) {
                const int kk = kc + b_k + e;
                rb[e] = (b_row_ok && kk < w) ? b_src[kk] : T(0);
            }
        } else {
            const int kk = kc + b_k;
#pragma unroll
            for (int e = 0; e < BPT; ++e) {
                const int c = col0 + b_c + e;
                rb[e] = (kk < w && c < n) ? b_src[idx(kc + b_k, e, lda)] : T(0);
            }
        }
    };
    auto store_chunk = [&](int buf) {
#pragma unroll
        for (int e = 0; e < APT; ++e) As[buf][a_k + e][a_r] = ra[e];
#pragma unroll
        for (int e = 0; e < BPT; ++e) {
            if (SYRK)
                Bs[buf][b_k + e][b_c] = rb[e];
            else
                Bs[buf][b_k][b_c + e] = rb[e];
        }
    };

    const int nchunk = cdiv(w, BK);
    load_chunk(0);
    store_chunk(0);
    __syncthreads();
    for (int ch = 0; ch < nchunk; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nchunk) load_chunk((ch + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(-av[i], bv[j], acc[i][j]);
        }
        if (ch + 1 < nchunk) store_chunk(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < m && c < n && (!SYRK || r >= c)) A[idx(r, c, lda)] = acc[i][j];
        }
}

int schur_f64(double* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = m - k - w, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    // The DFMA pipe (about 2 FMA/clk/SM) is the bound at any tile size; 64 x 64
    // tiles keep 88 registers per thread, two CTAs per SM and a short tail.
    dim3 grid(cdiv(N, 64), cdiv(M, 64));
    {
        ProfScope ps(LU_PROF_SCHUR, s, 2.0 * M * N * w, 8.0 * (2.0 * M * N + static_cast<double>(M + N) * w));
        schur_simt_kernel<double, 64, 64><<<grid, 256, 0, s>>>(A, lda, m, k, w, c0, c1);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// binary32 CUDA-core variant (the all-fp32 factorization): 128 x 128 tiles,
// 8 x 8 accumulators per thread.
int schur_f32(float* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = m - k - w, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    const long long big = static_cast<long long>(cdiv(M, 128)) * cdiv(N, 128);
    {
        ProfScope ps(LU_PROF_SCHUR, s, 2.0 * M * N * w, 4.0 * (2.0 * M * N + static_cast<double>(M + N) * w));
        if (big >= 152) {
            dim3 grid(cdiv(N, 128), cdiv(M, 128));
            schur_simt_kernel<float, 128, 128><<<grid, 256, 0, s>>>(A, lda, m, k, w, c0, c1);
        } else {
            dim3 grid(cdiv(N, 64), cdiv(M, 64));
            schur_simt_kernel<float, 64, 64><<<grid, 256, 0, s>>>(A, lda, m, k, w, c0, c1);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// Cholesky trailing update: the lower triangle of rows [c0, n) x columns
// [c0, c1) -= A[:, k:k+w) A[:, k:k+w)^T.  c1 == n is the whole trailing
// square (triangular tile grid); c1 < n is a panel of columns.
template <typename T>
int syrk_lower(T* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = n - c0, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    // lower elements of the region: columns c in [c0, c1) hold n - c each
    const double elems = static_cast<double>(N) * M - 0.5 * static_cast<double>(N) * (N - 1);
    constexpr int kElem = sizeof(T);
    // binary64: 64 x 64 tiles as in the LU update; binary32: 128 x 128 when
    // there are enough of them
    const bool big = sizeof(T) == 4 && static_cast<long long>(cdiv(M, 128)) * cdiv(N, 128) >= 152;
    const long long ntri = big ? static_cast<long long>(cdiv(M, 128)) * (cdiv(M, 128) + 1) / 2
                               : static_cast<long long>(cdiv(M, 64)) * (cdiv(M, 64) + 1) / 2;
    if (c1 == n && ntri > 0x7fffffffLL) return LU_EUNSUPPORTED;
    {
        ProfScope ps(LU_PROF_SYRK, s, 2.0 * elems * w, kElem * (2.0 * elems + static_cast<double>(M + N) * w));
        constexpr int BIG = sizeof(T) == 4 ? 128 : 64;     // binary64 never takes 128 x 128 tiles
        if (c1 == n) {
            const unsigned tiles = static_cast<unsigned>(ntri);
            if (big)
                schur_simt_kernel<T, BIG, BIG, true, true><<<tiles, 256, 0, s>>>(A, lda, n, k, w, c0, n);
            else
                schur_simt_kernel<T, 64, 64, true, true><<<tiles, 256, 0, s>>>(A, lda, n, k, w, c0, n);
        } else {
            if (big)
                schur_simt_kernel<T, BIG, BIG, true, false>
                    <<<dim3(cdiv(N, BIG), cdiv(M, BIG)), 256, 0, s>>>(A, lda, n, k, w, c0, c1);
            else
                schur_simt_kernel<T, 64, 64, true, false>
                    <<<dim3(cdiv(N, 64), cdiv(M, 64)), 256, 0, s>>>(A, lda, n, k, w, c0, c1);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template int syrk_lower<double>(double*, int, int, int, int, int, int, cudaStream_t);
template int syrk_lower<float>(float*, int, int, int, int, int, int, cudaStream_t);

}  // namespace lu
