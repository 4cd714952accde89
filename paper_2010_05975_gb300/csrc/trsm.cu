// FactorizeA10 and FactorizeA01 of Section 7.2 (binary64 or binary32):
//   L21 = A21 * U00^{-1}   (rows below the panel, right solve, upper U00;
//                           with U00 = L00^T also the Cholesky panel solve)
//   U12 = L00^{-1} * A12   (rows of the panel, left solve, unit lower L00)
// Every element receives its fused updates in ascending pivot order and then
// (L21 only) one IEEE division: the same operation sequence as the
// column-by-column and row-by-row forms of the definition, whichever kernel
// runs.  Rows of L21 (columns of U12) are independent, so the binary32
// kernels give each thread one row (column) and sweep it left-looking in
// register blocks against the triangle staged in shared memory: no barrier
// between steps.  The binary64 kernels, bound by the DFMA pipe, keep the
// right-looking sweep with four threads per row (column).
#include "common.cuh"
#include "prof.cuh"

namespace lu {

constexpr int kL21Rows = 64;      // rows of A21 per CTA
constexpr int kL21Stride = kL21Rows + 1;
constexpr int kU12Cols = 64;      // columns of A12 per CTA

// Tile T[j][r] (column-major over the CTA's rows, padded stride).  Thread t
// owns row r = t % 64 and columns c = j+1+g, j+1+g+4, ... with g = t / 64.
// U (w x w, row stride ldu) is read on and above its diagonal only: the LU
// passes A00 in place, the Cholesky factorization L00^T.
template <typename E>
__global__ void __launch_bounds__(256) trsm_l21_kernel(E* __restrict__ A, int lda, int m, int k, int w,
                                                       const E* __restrict__ U, int ldu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* T = reinterpret_cast<E*>(smem_raw);
    const int r0 = k + w + blockIdx.x * kL21Rows;
    const int nrow = min(kL21Rows, m - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = warp; r < kL21Rows; r += nwarp) {
        const bool ok = r < nrow;
        for (int j = lane; j < w; j += 32) T[j * kL21Stride + r] = ok ? A[idx(r0 + r, k + j, lda)] : E(0);
    }
    __syncthreads();
    const int r = threadIdx.x % kL21Rows, g = threadIdx.x / kL21Rows;
    for (int j = 0; j < w; ++j) {
        const E* Uj = U + idx(j, 0, ldu);
        if (g == 0) {
            const E u = Uj[j];
            const E a = T[j * kL21Stride + r];
            T[j * kL21Stride + r] = (u != E(0)) ? a / u : E(0);
        }
        __syncthreads();
        const E x = T[j * kL21Stride + r];
        for (int c = j + 1 + g; c < w; c += 4) T[c * kL21Stride + r] = fma(-x, Uj[c], T[c * kL21Stride + r]);
        __syncthreads();
    }
    for (int rr = warp; rr < nrow; rr += nwarp)
        for (int j = lane; j < w; j += 32) A[idx(r0 + rr, k + j, lda)] = T[j * kL21Stride + rr];
}

// Tile T[i][c] (row-major, w rows x 64 columns).  Thread t owns column
// c = t % 64 and rows i = p+1+g, p+1+g+4, ... with g = t / 64.
template <typename E>
__global__ void __launch_bounds__(256) trsm_u12_kernel(E* __restrict__ A, int lda, int n, int k, int w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* T = reinterpret_cast<E*>(smem_raw);
    const int c0 = k + w + blockIdx.x * kU12Cols;
    const int ncol = min(kU12Cols, n - c0);
    const int c = threadIdx.x % kU12Cols, g = threadIdx.x / kU12Cols;
    for (int i = g; i < w; i += 4) T[i * kU12Cols + c] = (c < ncol) ? A[idx(k + i, c0 + c, lda)] : E(0);
    __syncthreads();
    for (int p = 0; p + 1 < w; ++p) {
        const E up = T[p * kU12Cols + c];
        for (int i = p + 1 + g; i < w; i += 4)
            T[i * kU12Cols + c] = fma(-A[idx(k + i, k + p, lda)], up, T[i * kU12Cols + c]);
        __syncthreads();
    }
    if (c < ncol)
        for (int i = g; i < w; i += 4) A[idx(k + i, c0 + c, lda)] = T[i * kU12Cols + c];
}

// ---------------------------------------------------------------------------
// binary32: one thread per row (column), left-looking in register blocks.
// ---------------------------------------------------------------------------
constexpr int kRowCta = 64;        // rows of A21 (columns of A12) per CTA, one per thread
constexpr int kTileStride = kRowCta + 1;
constexpr int kStrip = 64;         // triangle columns (rows) staged per strip
constexpr int kStripStride = kStrip + 4;   // 16-byte rows; staging writes spread over banks
constexpr int kRb = 16;            // register block

__host__ __device__ constexpr int trsm_wp(int w) { return (w + kRb - 1) / kRb * kRb; }

// Shared memory: the strip S[j][c'] (stride kStripStride) then the tile
// T[j][r] (stride kTileStride, wp rows).
inline size_t trsm_rows_smem(int w) {
    return (static_cast<size_t>(w) * kStripStride + static_cast<size_t>(trsm_wp(w)) * kTileStride) * sizeof(float);
}

// acc[i] = fma(-x, v[i], acc[i]) for one register block, v 16-byte aligned.
__device__ __forceinline__ void trsm_axpy16(float (&acc)[kRb], float x, const float* v) {
#pragma unroll
    for (int q = 0; q < kRb / 4; ++q) {
        const float4 u = *reinterpret_cast<const float4*>(v + 4 * q);
        acc[4 * q + 0] = fmaf(-x, u.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(-x, u.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(-x, u.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(-x, u.w, acc[4 * q + 3]);
    }
}

// L21 = A21 * U^{-1}.  Thread r owns row r0 + r; its solved values replace
// the tile's in place.  Per strip of kStrip columns [s0, s1) the CTA stages
// U[0:s1, s0:s1) (upper part; zeros below the diagonal), then each thread
// takes its row's register blocks of the strip: the updates of every earlier
// column j (from the tile), then the block's own columns in order, each
// finished by its division.  Per element that is fma over j ascending, then
// the division: the sequence of the right-looking sweep.
__global__ void __launch_bounds__(kRowCta) trsm_l21_rows_kernel(float* __restrict__ A, int lda, int m, int k, int w,
                                                                const float* __restrict__ U, int ldu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* S = reinterpret_cast<float*>(smem_raw);
    float* T = S + static_cast<size_t>(w) * kStripStride;
    const int wp = trsm_wp(w);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = k + w + blockIdx.x * kRowCta;
    const int nrow = min(kRowCta, m - r0);
    for (int r = warp; r < kRowCta; r += kRowCta / 32) {
        const bool ok = r < nrow;
        for (int j = lane; j < wp; j += 32)
            T[j * kTileStride + r] = (ok && j < w) ? A[idx(r0 + r, k + j, lda)] : 0.f;
    }
    for (int s0 = 0; s0 < w; s0 += kStrip) {
        const int s1 = min(s0 + kStrip, w);
        __syncthreads();                                   // the previous strip is no longer read
        for (int e = tid; e < s1 * kStrip; e += kRowCta) {
            const int j = e / kStrip, c = s0 + e % kStrip;
            S[j * kStripStride + (c - s0)] = (c < s1 && c >= j) ? U[idx(j, c, ldu)] : 0.f;
        }
        __syncthreads();
        for (int c0 = s0; c0 < s1; c0 += kRb) {
            float acc[kRb];
#pragma unroll
            for (int i = 0; i < kRb; ++i) acc[i] = T[(c0 + i) * kTileStride + tid];
#pragma unroll 4
            for (int j = 0; j < c0; ++j) trsm_axpy16(acc, T[j * kTileStride + tid], S + j * kStripStride + (c0 - s0));
#pragma unroll
            for (int jj = 0; jj < kRb; ++jj) {
                if (c0 + jj < s1) {
                    const float* Sj = S + (c0 + jj) * kStripStride + (c0 - s0);
                    const float u = Sj[jj];
                    acc[jj] = (u != 0.f) ? acc[jj] / u : 0.f;
#pragma unroll
                    for (int i = jj + 1; i < kRb; ++i) acc[i] = fmaf(-acc[jj], Sj[i], acc[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < kRb; ++i) T[(c0 + i) * kTileStride + tid] = acc[i];
        }
    }
    __syncthreads();
    for (int r = warp; r < nrow; r += kRowCta / 32)
        for (int j = lane; j < w; j += 32) A[idx(r0 + r, k + j, lda)] = T[j * kTileStride + r];
}

// U12 = L00^{-1} * A12 (unit lower L00 = the strict lower part of the
// diagonal block).  Thread c owns column c0 + c.  Per strip of kStrip rows
// [s0, s1) the CTA stages L00[s0:s1, 0:s1) transposed, S[p][i - s0] =
// L(i, p) for p < i (zeros elsewhere), then each thread takes its column's
// register blocks of the strip: the updates of every earlier row p, then the
// block's own rows in order.  Per element: fma over p ascending.
__global__ void __launch_bounds__(kRowCta) trsm_u12_cols_kernel(float* __restrict__ A, int lda, int n, int k, int w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* S = reinterpret_cast<float*>(smem_raw);
    float* T = S + static_cast<size_t>(w) * kStripStride;    // T[i][c], stride kTileStride
    const int wp = trsm_wp(w);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cb = k + w + blockIdx.x * kRowCta;
    const int ncol = min(kRowCta, n - cb);
    for (int i = warp; i < wp; i += kRowCta / 32)
        for (int c = lane; c < kRowCta; c += 32)
            T[i * kTileStride + c] = (i < w && c < ncol) ? A[idx(k + i, cb + c, lda)] : 0.f;
    for (int s0 = 0; s0 < w; s0 += kStrip) {
        const int s1 = min(s0 + kStrip, w);
        __syncthreads();
        for (int e = tid; e < kStrip * s1; e += kRowCta) {
            const int ii = e / s1, p = e - ii * s1;       // row s0 + ii of L00, coalesced along p
            const int i = s0 + ii;
            S[p * kStripStride + ii] = (i < s1 && p < i) ? A[idx(k + i, k + p, lda)] : 0.f;
        }
        __syncthreads();
        for (int i0 = s0; i0 < s1; i0 += kRb) {
            float acc[kRb];
#pragma unroll
            for (int i = 0; i < kRb; ++i) acc[i] = T[(i0 + i) * kTileStride + tid];
#pragma unroll 4
            for (int p = 0; p < i0; ++p) trsm_axpy16(acc, T[p * kTileStride + tid], S + p * kStripStride + (i0 - s0));
#pragma unroll
            for (int pp = 0; pp + 1 < kRb; ++pp) {
                if (i0 + pp < s1) {
                    const float* Sp = S + (i0 + pp) * kStripStride + (i0 - s0);
#pragma unroll
                    for (int i = pp + 1; i < kRb; ++i) acc[i] = fmaf(-Sp[i], acc[pp], acc[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < kRb; ++i) T[(i0 + i) * kTileStride + tid] = acc[i];
        }
    }
    __syncthreads();
    for (int i = warp; i < w; i += kRowCta / 32)
        for (int c = lane; c < ncol; c += 32) A[idx(k + i, cb + c, lda)] = T[i * kTileStride + c];
}

template <typename E>
int trsm_l21(E* A, int lda, int m, int k, int w, const E* U, int ldu, cudaStream_t s) {
    const int rows = m - k - w;
    if (rows <= 0) return 0;
    ProfScope ps(LU_PROF_TRSM_L21, s, static_cast<double>(rows) * w * w);
    if constexpr (sizeof(E) == 4) {
        const size_t smem = trsm_rows_smem(w);
        if (int rc_ = smem_attr(trsm_l21_rows_kernel, smem)) return rc_;
        trsm_l21_rows_kernel<<<cdiv(rows, kRowCta), kRowCta, smem, s>>>(A, lda, m, k, w, U, ldu);
    } else {
        const size_t smem = static_cast<size_t>(w) * kL21Stride * sizeof(E);
        if (int rc_ = smem_attr(trsm_l21_kernel<E>, smem)) return rc_;
        trsm_l21_kernel<E><<<cdiv(rows, kL21Rows), 256, smem, s>>>(A, lda, m, k, w, U, ldu);
    }
    count_launches(1);
    LU_LAUNCHED();
    return 0;
}

template <typename E>
int trsm_u12(E* A, int lda, int n, int k, int w, cudaStream_t s) {
    const int cols = n - k - w;
    if (cols <= 0 || w <= 1) return 0;
    ProfScope ps(LU_PROF_TRSM_U12, s, static_cast<double>(cols) * w * (w - 1));
    if constexpr (sizeof(E) == 4) {
        const size_t smem = trsm_rows_smem(w);
        if (int rc_ = smem_attr(trsm_u12_cols_kernel, smem)) return rc_;
        trsm_u12_cols_kernel<<<cdiv(cols, kRowCta), kRowCta, smem, s>>>(A, lda, n, k, w);
    } else {
        const size_t smem = static_cast<size_t>(w) * kU12Cols * sizeof(E);
        if (int rc_ = smem_attr(trsm_u12_kernel<E>, smem)) return rc_;
        trsm_u12_kernel<E><<<cdiv(cols, kU12Cols), 256, smem, s>>>(A, lda, n, k, w);
    }
    count_launches(1);
    LU_LAUNCHED();
    return 0;
}

template int trsm_l21<double>(double*, int, int, int, int, const double*, int, cudaStream_t);
template int trsm_l21<float>(float*, int, int, int, int, const float*, int, cudaStream_t);
template int trsm_u12<double>(double*, int, int, int, int, cudaStream_t);
template int trsm_u12<float>(float*, int, int, int, int, cudaStream_t);

}  // namespace lu
