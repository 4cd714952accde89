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
// right-looking sweep with eight threads per row (column).
#include "common.cuh"
#include "prof.cuh"

namespace lu {

// Rows of A21 (columns of A12) per CTA of 256 threads: 32 in binary64, so
// that a 256-wide panel's tile (64 KB) lets three CTAs share an SM and the
// late steps' short blocks still spread over every SM; 64 in binary32.
template <typename E>
__host__ __device__ constexpr int trsm_tile_rows() { return sizeof(E) == 8 ? 32 : 64; }

// Tile T[j][r] (column-major over the CTA's R rows, padded stride R + 1).
// Thread t owns row r = t % R and columns c = j+1+g, j+1+g+G, ... with
// g = t / R and G = 256 / R.  U (w x w, row stride ldu) is read on and above
// its diagonal only: the LU passes A00 in place, the Cholesky factorization
// L00^T.
template <typename E>
__global__ void __launch_bounds__(256) trsm_l21_kernel(E* __restrict__ A, int lda, int m, int k, int w,
                                                       const E* __restrict__ U, int ldu) {
    constexpr int R = trsm_tile_rows<E>(), G = 256 / R, ST = R + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* T = reinterpret_cast<E*>(smem_raw);
    const int r0 = k + w + blockIdx.x * R;
    const int nrow = min(R, m - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = warp; r < R; r += nwarp) {
        const bool ok = r < nrow;
        for (int j = lane; j < w; j += 32) T[j * ST + r] = ok ? A[idx(r0 + r, k + j, lda)] : E(0);
    }
    __syncthreads();
    const int r = threadIdx.x % R, g = threadIdx.x / R;
    for (int j = 0; j < w; ++j) {
        const E* Uj = U + idx(j, 0, ldu);
        if (g == 0) {
            const E u = Uj[j];
            const E a = T[j * ST + r];
            T[j * ST + r] = (u != E(0)) ? a / u : E(0);
        }
        __syncthreads();
        const E x = T[j * ST + r];
        for (int c = j + 1 + g; c < w; c += G) T[c * ST + r] = fma(-x, Uj[c], T[c * ST + r]);
        __syncthreads();
    }
    for (int rr = warp; rr < nrow; rr += nwarp)
        for (int j = lane; j < w; j += 32) A[idx(r0 + rr, k + j, lda)] = T[j * ST + rr];
}

// Tile T[i][c] (row-major, w rows x C columns, C = trsm_tile_rows).  Thread
// t owns column c = t % C and rows i = p+1+g, p+1+g+G, ... with g = t / C.
template <typename E>
__global__ void __launch_bounds__(256) trsm_u12_kernel(E* __restrict__ A, int lda, int n, int k, int w) {
    constexpr int C = trsm_tile_rows<E>(), G = 256 / C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* T = reinterpret_cast<E*>(smem_raw);
    const int c0 = k + w + blockIdx.x * C;
    const int ncol = min(C, n - c0);
    const int c = threadIdx.x % C, g = threadIdx.x / C;
    for (int i = g; i < w; i += G) T[i * C + c] = (c < ncol) ? A[idx(k + i, c0 + c, lda)] : E(0);
    __syncthreads();
    for (int p = 0; p + 1 < w; ++p) {
        const E up = T[p * C + c];
        for (int i = p + 1 + g; i < w; i += G) T[i * C + c] = fma(-A[idx(k + i, k + p, lda)], up, T[i * C + c]);
        __syncthreads();
    }
    if (c < ncol)
        for (int i = g; i < w; i += G) A[idx(k + i, c0 + c, lda)] = T[i * C + c];
}

// ---------------------------------------------------------------------------
// binary32: one thread per row (column), left-looking in register blocks.
// ---------------------------------------------------------------------------
constexpr int kRowCta = 64;        // rows of A21 (columns of A12) per CTA, one per thread
constexpr int kStrip = 64;         // triangle columns (rows) staged per strip
constexpr int kRb = 16;            // register block

__host__ __device__ constexpr int trsm_wp(int w) { return (w + kRb - 1) / kRb * kRb; }
// Row pitches (floats): a whole number of 16-byte chunks plus one, so that
// eight consecutive rows' 16-byte reads fall in distinct bank groups.
__host__ __device__ constexpr int trsm_pitch(int cols) { return (cols + 3) / 4 * 4 + 4; }

// Shared memory: the tile (kRowCta rows of wp columns for L21, wp rows of
// kRowCta columns for U12) and one strip of the triangle.
inline size_t trsm_l21_smem(int w) {
    return (static_cast<size_t>(kRowCta) * trsm_pitch(trsm_wp(w)) +
            static_cast<size_t>(w) * trsm_pitch(kStrip)) * sizeof(float);
}
inline size_t trsm_u12_smem(int w) {
    return (static_cast<size_t>(trsm_wp(w)) * trsm_pitch(kRowCta) +
            static_cast<size_t>(kStrip) * trsm_pitch(trsm_wp(w))) * sizeof(float);
}

// Stage rows x cols of a row-major global block (leading dimension ld) into
// shared memory (pitch floats per row), zero outside [0, vrows) x [0, vcols).
// vec: the global rows start 16-byte aligned, so 16-byte asynchronous copies
// are used; otherwise plain loads.
__device__ __forceinline__ void trsm_stage(float* dst, int pitch, const float* src, size_t ld, int rows, int cols,
                                           int vrows, int vcols, bool vec) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (vec) {
        const int cq = (cols + 3) / 4;
        for (int e = tid; e < rows * cq; e += nt) {
            const int r = e / cq, c = 4 * (e - r * cq);
            const int bytes = (r < vrows) ? 4 * max(0, min(4, vcols - c)) : 0;
            cp_async16(dst + static_cast<size_t>(r) * pitch + c, bytes ? src + r * ld + c : src, bytes);
        }
        cp_async_wait_all();
    } else {
        for (int e = tid; e < rows * cols; e += nt) {
            const int r = e / cols, c = e - r * cols;
            dst[static_cast<size_t>(r) * pitch + c] = (r < vrows && c < vcols) ? src[r * ld + c] : 0.f;
        }
    }
}

// acc[i] = fma(-x[q], v_q[i], acc[i]) for q = 0..3 in order, v_q = v + q * vp
// (16-byte aligned rows of the staged triangle).
__device__ __forceinline__ void trsm_axpy16x4(float (&acc)[kRb], const float4 x, const float* v, int vp) {
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int h = 0; h < kRb / 4; ++h) {
            const float4 u = *reinterpret_cast<const float4*>(v + q * vp + 4 * h);
            acc[4 * h + 0] = fmaf(-xs[q], u.x, acc[4 * h + 0]);
            acc[4 * h + 1] = fmaf(-xs[q], u.y, acc[4 * h + 1]);
            acc[4 * h + 2] = fmaf(-xs[q], u.z, acc[4 * h + 2]);
            acc[4 * h + 3] = fmaf(-xs[q], u.w, acc[4 * h + 3]);
        }
    }
}

// L21 = A21 * U^{-1}.  Thread r owns row r0 + r, kept in the tile T[r][j]
// (row-major), whose solved values replace the inputs in place.  Per strip
// of kStrip columns [s0, s1) the CTA stages U[0:s1, s0:s1) (only entries on
// or above the diagonal are read), then each thread takes its row's
// register blocks of the strip: the updates of every earlier column j, four
// at a time from one 16-byte read of its row, then the block's own columns
// in order, each finished by its division.  Per element that is fma over j
// ascending, then the division: the sequence of the right-looking sweep.
__global__ void __launch_bounds__(kRowCta) trsm_l21_rows_kernel(float* __restrict__ A, int lda, int m, int k, int w,
                                                                const float* __restrict__ U, int ldu, int vec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wp = trsm_wp(w);
    const int tp = trsm_pitch(wp), sp = trsm_pitch(kStrip);
    float* T = reinterpret_cast<float*>(smem_raw);
    float* S = T + static_cast<size_t>(kRowCta) * tp;
    const int tid = threadIdx.x;
    const int r0 = k + w + blockIdx.x * kRowCta;
    const int nrow = min(kRowCta, m - r0);
    trsm_stage(T, tp, A + idx(r0, k, lda), lda, kRowCta, wp, nrow, w, vec != 0);
    float* Tr = T + static_cast<size_t>(tid) * tp;
    for (int s0 = 0; s0 < w; s0 += kStrip) {
        const int s1 = min(s0 + kStrip, w);
        __syncthreads();                                   // the tile is in; the previous strip is no longer read
        trsm_stage(S, sp, U + idx(0, s0, ldu), ldu, s1, kStrip, s1, s1 - s0, vec != 0);
        __syncthreads();
        for (int c0 = s0; c0 < s1; c0 += kRb) {
            float acc[kRb];
#pragma unroll
            for (int i = 0; i < kRb; i += 4) {
                const float4 v = *reinterpret_cast<const float4*>(Tr + c0 + i);
                acc[i] = v.x;
                acc[i + 1] = v.y;
                acc[i + 2] = v.z;
                acc[i + 3] = v.w;
            }
#pragma unroll 2
            for (int j = 0; j < c0; j += 4)
                trsm_axpy16x4(acc, *reinterpret_cast<const float4*>(Tr + j), S + j * sp + (c0 - s0), sp);
#pragma unroll
            for (int jj = 0; jj < kRb; ++jj) {
                if (c0 + jj < s1) {
                    const float* Sj = S + (c0 + jj) * sp + (c0 - s0);
                    const float u = Sj[jj];
                    acc[jj] = (u != 0.f) ? acc[jj] / u : 0.f;
#pragma unroll
                    for (int i = jj + 1; i < kRb; ++i) acc[i] = fmaf(-acc[jj], Sj[i], acc[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < kRb; i += 4)
                *reinterpret_cast<float4*>(Tr + c0 + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
        }
    }
    __syncthreads();
    for (int e = tid; e < nrow * w; e += kRowCta) {
        const int r = e / w, j = e - r * w;
        A[idx(r0 + r, k + j, lda)] = T[static_cast<size_t>(r) * tp + j];
    }
}

// U12 = L00^{-1} * A12 (unit lower L00 = the strict lower part of the
// diagonal block).  Thread c owns column cb + c of the tile T[i][c].  Per
// strip of kStrip rows [s0, s1) the CTA stages rows s0..s1-1 of L00
// (columns 0..s1-1; only entries left of the diagonal are read), then each
// thread takes its column's register blocks of the strip: the updates of
// every earlier row p, four at a time (one 16-byte read of L per row of the
// block), then the block's own rows in order.  Per element: fma over p
// ascending.
__global__ void __launch_bounds__(kRowCta) trsm_u12_cols_kernel(float* __restrict__ A, int lda, int n, int k, int w,
                                                                int vec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wp = trsm_wp(w);
    const int tp = trsm_pitch(kRowCta), sp = trsm_pitch(wp);
    float* T = reinterpret_cast<float*>(smem_raw);
    float* S = T + static_cast<size_t>(wp) * tp;
    const int tid = threadIdx.x;
    const int cb = k + w + blockIdx.x * kRowCta;
    const int ncol = min(kRowCta, n - cb);
    trsm_stage(T, tp, A + idx(k, cb, lda), lda, wp, kRowCta, w, ncol, vec != 0);
    for (int s0 = 0; s0 < w; s0 += kStrip) {
        const int s1 = min(s0 + kStrip, w);
        __syncthreads();
        trsm_stage(S, sp, A + idx(k + s0, k, lda), lda, kStrip, wp, s1 - s0, s1, vec != 0);
        __syncthreads();
        for (int i0 = s0; i0 < s1; i0 += kRb) {
            const float* Sb = S + static_cast<size_t>(i0 - s0) * sp;   // row i0 of L00
            float acc[kRb];
#pragma unroll
            for (int i = 0; i < kRb; ++i) acc[i] = T[(i0 + i) * tp + tid];
#pragma unroll 2
            for (int p = 0; p < i0; p += 4) {
                const float x0 = T[p * tp + tid], x1 = T[(p + 1) * tp + tid];
                const float x2 = T[(p + 2) * tp + tid], x3 = T[(p + 3) * tp + tid];
#pragma unroll
                for (int i = 0; i < kRb; ++i) {
                    const float4 l = *reinterpret_cast<const float4*>(Sb + i * sp + p);
                    acc[i] = fmaf(-l.x, x0, acc[i]);
                    acc[i] = fmaf(-l.y, x1, acc[i]);
                    acc[i] = fmaf(-l.z, x2, acc[i]);
                    acc[i] = fmaf(-l.w, x3, acc[i]);
                }
            }
#pragma unroll
            for (int pp = 0; pp + 1 < kRb; ++pp) {
                if (i0 + pp < s1) {
#pragma unroll
                    for (int i = pp + 1; i < kRb; ++i) acc[i] = fmaf(-Sb[i * sp + i0 + pp], acc[pp], acc[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < kRb; ++i) T[(i0 + i) * tp + tid] = acc[i];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < w; i += kRowCta / 32)
        for (int c = threadIdx.x & 31; c < ncol; c += 32) A[idx(k + i, cb + c, lda)] = T[i * tp + c];
}

// Panels wider than this much shared memory allows (w > 384) take the
// right-looking kernels above.
constexpr size_t kTrsmSmemMax = 200 * 1024;

// 16-byte asynchronous staging needs every staged row to start 16-byte
// aligned: the base and the leading dimension in whole 16-byte chunks.
inline int trsm_vec(const void* p, int ld) {
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld & 3) == 0) ? 1 : 0;
}

template <typename E>
int trsm_l21(E* A, int lda, int m, int k, int w, const E* U, int ldu, cudaStream_t s) {
    const int rows = m - k - w;
    if (rows <= 0) return 0;
    ProfScope ps(LU_PROF_TRSM_L21, s, static_cast<double>(rows) * w * w);
    bool done = false;
    if constexpr (sizeof(E) == 4) {
        const size_t smem = trsm_l21_smem(w);
        if (smem <= kTrsmSmemMax) {
            if (int rc_ = smem_attr(trsm_l21_rows_kernel, smem)) return rc_;
            const int vec = trsm_vec(A + idx(k + w, k, lda), lda) & trsm_vec(U, ldu);
            trsm_l21_rows_kernel<<<cdiv(rows, kRowCta), kRowCta, smem, s>>>(A, lda, m, k, w, U, ldu, vec);
            done = true;
        }
    }
    if (!done) {
        constexpr int R = trsm_tile_rows<E>();
        const size_t smem = static_cast<size_t>(w) * (R + 1) * sizeof(E);
        if (int rc_ = smem_attr(trsm_l21_kernel<E>, smem)) return rc_;
        trsm_l21_kernel<E><<<cdiv(rows, R), 256, smem, s>>>(A, lda, m, k, w, U, ldu);
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
    bool done = false;
    if constexpr (sizeof(E) == 4) {
        const size_t smem = trsm_u12_smem(w);
        if (smem <= kTrsmSmemMax) {
            if (int rc_ = smem_attr(trsm_u12_cols_kernel, smem)) return rc_;
            const int vec = trsm_vec(A + idx(k, k + w, lda), lda) & trsm_vec(A + idx(k, k, lda), lda);
            trsm_u12_cols_kernel<<<cdiv(cols, kRowCta), kRowCta, smem, s>>>(A, lda, n, k, w, vec);
            done = true;
        }
    }
    if (!done) {
        constexpr int C = trsm_tile_rows<E>();
        const size_t smem = static_cast<size_t>(w) * C * sizeof(E);
        if (int rc_ = smem_attr(trsm_u12_kernel<E>, smem)) return rc_;
        trsm_u12_kernel<E><<<cdiv(cols, C), 256, smem, s>>>(A, lda, n, k, w);
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
