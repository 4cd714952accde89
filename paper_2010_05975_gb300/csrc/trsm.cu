// FactorizeA10 and FactorizeA01 of Section 7.2 (binary64 or binary32):
//   L21 = A21 * U00^{-1}   (rows below the panel, right solve, upper U00;
//                           with U00 = L00^T also the Cholesky panel solve)
//   U12 = L00^{-1} * A12   (rows of the panel, left solve, unit lower L00)
// Both keep a tile in shared memory and sweep the triangle right-looking,
// so every element receives its fused updates in ascending pivot order and
// then (L21 only) one IEEE division: the same operation sequence as the
// column-by-column and row-by-row forms of the definition.
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

template <typename E>
int trsm_l21(E* A, int lda, int m, int k, int w, const E* U, int ldu, cudaStream_t s) {
    const int rows = m - k - w;
    if (rows <= 0) return 0;
    const size_t smem = static_cast<size_t>(w) * kL21Stride * sizeof(E);
    if (int rc_ = smem_attr(trsm_l21_kernel<E>, smem)) return rc_;
    {
        ProfScope ps(LU_PROF_TRSM_L21, s, static_cast<double>(rows) * w * w);
        trsm_l21_kernel<E><<<cdiv(rows, kL21Rows), 256, smem, s>>>(A, lda, m, k, w, U, ldu);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template <typename E>
int trsm_u12(E* A, int lda, int n, int k, int w, cudaStream_t s) {
    const int cols = n - k - w;
    if (cols <= 0 || w <= 1) return 0;
    const size_t smem = static_cast<size_t>(w) * kU12Cols * sizeof(E);
    if (int rc_ = smem_attr(trsm_u12_kernel<E>, smem)) return rc_;
    {
        ProfScope ps(LU_PROF_TRSM_U12, s, static_cast<double>(cols) * w * (w - 1));
        trsm_u12_kernel<E><<<cdiv(cols, kU12Cols), 256, smem, s>>>(A, lda, n, k, w);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template int trsm_l21<double>(double*, int, int, int, int, const double*, int, cudaStream_t);
template int trsm_l21<float>(float*, int, int, int, int, const float*, int, cudaStream_t);
template int trsm_u12<double>(double*, int, int, int, int, cudaStream_t);
template int trsm_u12<float>(float*, int, int, int, int, cudaStream_t);

}  // namespace lu
