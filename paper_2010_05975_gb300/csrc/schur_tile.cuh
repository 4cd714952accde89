// Register-tiled update kernel shared by the binary64 and binary32 paths:
// A22 -= L21 * U12 (FactorizeA11, Section 7.2) and, instantiated with SYRK,
// the lower-triangle update -= L21 * L21^T of the Cholesky factorization.
//
// A CTA tile of BM x BN outputs, 256 threads, TM x TN accumulators per
// thread, K staged through shared memory in double-buffered chunks of 8.
// Each accumulator starts from the A22 value and receives fma(-l, u, acc)
// for p = 0, 1, ..., w-1, the oracle's order, so the result is bit-identical
// to it.  With SYRK the lower triangle (r >= c) of rows [c0, m) x columns
// [c0, c1) is updated, both operands read from the rows of L21 (columns
// [k, k+w)); TRI enumerates only the tiles of the square's lower triangle
// (c1 = m); without it the grid is a rectangle (a panel of columns) and
// tiles wholly above the diagonal exit at once.
#pragma once
#include "common.cuh"

namespace lu {

// Tile (row0, col0) of a launch: the lower-triangle enumeration t =
// ti (ti + 1) / 2 + tj (tj <= ti) for SYRK && TRI, else the 2-D grid.
template <bool SYRK, bool TRI, int BM, int BN>
__device__ __forceinline__ void update_tile_origin(int k, int w, int c0, int& row0, int& col0) {
    if (SYRK && TRI) {
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
}

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
    update_tile_origin<SYRK, TRI, BM, BN>(k, w, c0, row0, col0);
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

}  // namespace lu
