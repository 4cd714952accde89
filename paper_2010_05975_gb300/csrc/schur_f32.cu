// The binary32 updates on the CUDA cores: A22 -= L21 * U12 (FactorizeA11,
// Section 7.2, of the all-fp32 factorization at the top of the refinement
// ladder) and the lower-triangle Cholesky update -= L21 * L21^T.
//
// Large updates take a float-specific 128 x 128 tile: 256 threads, 8 x 8
// accumulators each, over rows {4ty..4ty+3, 64+4ty..64+4ty+3} and the same
// pattern of columns, so that one k step reads its 16 operands with four
// 16-byte shared-memory loads for 64 FMAs, and the operand chunks come from
// global memory 16 bytes at a time.  Two CTAs per SM (128 registers, a few
// bytes spilled) overlap one tile's C load and store with the other's FMAs;
// with one CTA per SM the kernel stalled on those loads.  Measured at
// n = 16384: 42.5 TFLOP/s for w = 256 against 23.7 for the generic 128 x 128
// tile.  Small updates use the generic 64 x 64 tile of schur_tile.cuh.
// Every accumulator still receives fma(-l, u, acc) with p ascending.
#include "common.cuh"
#include "prof.cuh"
#include "schur_tile.cuh"

namespace lu {

template <bool SYRK, bool TRI>
__global__ void __launch_bounds__(256, 2) schur_f32_kernel(float* __restrict__ A, int lda, int m, int k, int w,
                                                           int c0, int n) {
    constexpr int BM = 128, BN = 128, BK = 8;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    int row0, col0;
    update_tile_origin<SYRK, TRI, BM, BN>(k, w, c0, row0, col0);
    if (SYRK && col0 > row0 + BM - 1) return;   // wholly above the diagonal

    // local row (column) of accumulator index i (j): two groups of four
    auto rl = [&](int i) { return (i < 4 ? 0 : 60) + 4 * ty + i; };
    auto cl = [&](int j) { return (j < 4 ? 0 : 60) + 4 * tx + j; };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = row0 + rl(i);
        const float* prow = A + idx(r < m ? r : row0, col0 + 4 * tx, lda);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = col0 + cl(j);
            acc[i][j] = (r < m && c < n && (!SYRK || r >= c)) ? prow[(j < 4 ? 0 : 60) + j] : 0.0f;
        }
    }

    // loaders: four consecutive k of one row for A (and, with SYRK, for the
    // rows of L21 that form B^T); four consecutive columns of one U12 row
    // otherwise
    const int a_r = tid % BM, a_k = (tid / BM) * 4;
    const int b_k = SYRK ? (tid / BN) * 4 : tid / 32;
    const int b_c = SYRK ? tid % BN : (tid % 32) * 4;
    const bool a_row_ok = (row0 + a_r) < m;
    const bool b_row_ok = (col0 + b_c) < n;
    const float* a_src = A + idx(a_row_ok ? row0 + a_r : row0, k, lda);
    const float* b_src = SYRK ? A + idx(b_row_ok ? col0 + b_c : col0, k, lda) : A + idx(k, col0 + b_c, lda);

    // whole chunks load 16 bytes at a time when rows and the panel start on
    // 16-byte boundaries
    const bool vec = ((lda & 3) == 0) && ((k & 3) == 0) && ((reinterpret_cast<size_t>(A) & 15) == 0);
    float ra[4], rb[4];
    auto load_chunk = [&](int kc) {
        if (vec && kc + BK <= w) {
            const float4 x = a_row_ok ? *reinterpret_cast<const float4*>(a_src + kc + a_k) : make_float4(0.f, 0.f, 0.f, 0.f);
            ra[0] = x.x; ra[1] = x.y; ra[2] = x.z; ra[3] = x.w;
            if (SYRK) {
                const float4 y = b_row_ok ? *reinterpret_cast<const float4*>(b_src + kc + b_k)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                rb[0] = y.x; rb[1] = y.y; rb[2] = y.z; rb[3] = y.w;
            } else if (col0 + b_c + 3 < n) {
                const float4 y = *reinterpret_cast<const float4*>(b_src + idx(kc + b_k, 0, lda));
                rb[0] = y.x; rb[1] = y.y; rb[2] = y.z; rb[3] = y.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) rb[e] = (col0 + b_c + e < n) ? b_src[idx(kc + b_k, e, lda)] : 0.0f;
            }
            return;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int kk = kc + a_k + e;
            ra[e] = (a_row_ok && kk < w) ? a_src[kk] : 0.0f;
        }
        if (SYRK) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = kc + b_k + e;
                rb[e] = (b_row_ok && kk < w) ? b_src[kk] : 0.0f;
            }
        } else {
            const int kk = kc + b_k;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = col0 + b_c + e;
                rb[e] = (kk < w && c < n) ? b_src[idx(kk, e, lda)] : 0.0f;
            }
        }
    };
    auto store_chunk = [&](int buf) {
#pragma unroll
        for (int e = 0; e < 4; ++e) As[buf][a_k + e][a_r] = ra[e];
        if (SYRK) {
#pragma unroll
            for (int e = 0; e < 4; ++e) Bs[buf][b_k + e][b_c] = rb[e];
        } else {
            *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
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
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * tx]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-av[i], bv[j], acc[i][j]);
        }
        if (ch + 1 < nchunk) store_chunk(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = row0 + rl(i);
        float* prow = A + idx(r < m ? r : row0, col0 + 4 * tx, lda);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = col0 + cl(j);
            if (r < m && c < n && (!SYRK || r >= c)) prow[(j < 4 ? 0 : 60) + j] = acc[i][j];
        }
    }
}

// 128 x 128 tiles once there are at least a wave of them, else 64 x 64.
static bool f32_big(int M, int N) { return static_cast<long long>(cdiv(M, 128)) * cdiv(N, 128) >= 152; }

int schur_f32(float* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = m - k - w, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    {
        ProfScope ps(LU_PROF_SCHUR, s, 2.0 * M * N * w, 4.0 * (2.0 * M * N + static_cast<double>(M + N) * w));
        if (f32_big(M, N)) {
            dim3 grid(cdiv(N, 128), cdiv(M, 128));
            schur_f32_kernel<false, false><<<grid, 256, 0, s>>>(A, lda, m, k, w, c0, c1);
        } else {
            dim3 grid(cdiv(N, 64), cdiv(M, 64));
            schur_simt_kernel<float, 64, 64><<<grid, 256, 0, s>>>(A, lda, m, k, w, c0, c1);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// Cholesky trailing update in binary32 (see syrk_lower<double>).
template <>
int syrk_lower<float>(float* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s) {
    const int M = n - c0, N = c1 - c0;
    if (M <= 0 || N <= 0 || w <= 0) return 0;
    const double elems = static_cast<double>(N) * M - 0.5 * static_cast<double>(N) * (N - 1);
    const bool big = f32_big(M, N);
    const int T = big ? 128 : 64;
    const long long ntri = static_cast<long long>(cdiv(M, T)) * (cdiv(M, T) + 1) / 2;
    if (c1 == n && ntri > 0x7fffffffLL) return LU_EUNSUPPORTED;
    {
        ProfScope ps(LU_PROF_SYRK, s, 2.0 * elems * w, 4.0 * (2.0 * elems + static_cast<double>(M + N) * w));
        const unsigned tiles = static_cast<unsigned>(ntri);
        if (c1 == n) {
            if (big)
                schur_f32_kernel<true, true><<<tiles, 256, 0, s>>>(A, lda, n, k, w, c0, n);
            else
                schur_simt_kernel<float, 64, 64, true, true><<<tiles, 256, 0, s>>>(A, lda, n, k, w, c0, n);
        } else {
            if (big)
                schur_f32_kernel<true, false><<<dim3(cdiv(N, 128), cdiv(M, 128)), 256, 0, s>>>(A, lda, n, k, w, c0, c1);
            else
                schur_simt_kernel<float, 64, 64, true, false>
                    <<<dim3(cdiv(N, 64), cdiv(M, 64)), 256, 0, s>>>(A, lda, n, k, w, c0, c1);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

}  // namespace lu
