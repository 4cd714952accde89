// FactorizeA11 (Section 7.2) in binary64: A22 -= L21 * U12, K = w <= 256,
// and the Cholesky update of the lower triangle.
//
// GB300 executes binary64 on the CUDA cores only (no tcgen05 kind for it;
// measured DFMA ~1.19 TFLOP/s per GPU, DMMA m8n8k4 slower), so both are the
// register-tiled DFMA kernel of schur_tile.cuh with 64 x 64 tiles: 4 x 4
// accumulators per thread, 88 registers, two CTAs per SM.
#include "common.cuh"
#include "prof.cuh"
#include "schur_tile.cuh"

namespace lu {

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

// Cholesky trailing update: the lower triangle of rows [c0, n) x columns
// [c0, c1) -= A[:, k:k+w) A[:, k:k+w)^T.  c1 == n is the whole trailing
// square (triangular tile grid); c1 < n is a panel of columns.
template <>
int syrk_lower<double>(double* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = n - c0, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    // lower elements of the region: columns c in [c0, c1) hold n - c each
    const double elems = static_cast<double>(N) * M - 0.5 * static_cast<double>(N) * (N - 1);
    const long long ntri = static_cast<long long>(cdiv(M, 64)) * (cdiv(M, 64) + 1) / 2;
    if (c1 == n && ntri > 0x7fffffffLL) return LU_EUNSUPPORTED;
    {
        ProfScope ps(LU_PROF_SYRK, s, 2.0 * elems * w, 8.0 * (2.0 * elems + static_cast<double>(M + N) * w));
        if (c1 == n)
            schur_simt_kernel<double, 64, 64, true, true>
                <<<static_cast<unsigned>(ntri), 256, 0, s>>>(A, lda, n, k, w, c0, n);
        else
            schur_simt_kernel<double, 64, 64, true, false>
                <<<dim3(cdiv(N, 64), cdiv(M, 64)), 256, 0, s>>>(A, lda, n, k, w, c0, c1);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

}  // namespace lu
