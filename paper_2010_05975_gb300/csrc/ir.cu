// Mixed-precision LU + binary64 iterative refinement (the paper factors; it
// does not refine -- this is the solver the low-precision factorization
// serves).  The factorization runs on a binary32 copy of A with bf16 / fp8 /
// fp32 Schur operands; every residual, backward error and solution update is
// binary64.
//
//   x0 = (float solve with the low-precision factors)
//   repeat: r = b - A x (fp64); eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf)
//           stop at eta <= tol;  d = LU^{-1} (r / ||r||) * ||r|| (fp32 solve);
//           up to J inner steps d += LU^{-1} (r - A d) with the products A d
//           in binary32 multiplies (matvec32_kernel), while the inner
//           residual keeps shrinking by 2x and stays above 1e-6 ||r||; x += d
// Once a classical step cuts eta by less than 4x, the correction equation
// A d = r is solved instead (for the rest of the solve) by
// right-preconditioned flexible GMRES (binary64 Arnoldi, preconditioner =
// the fp32 solve, classical Gram-Schmidt applied twice, restart m).  The
// Arnoldi products A z first use binary32 multiplies (matvec32_kernel): the
// correction equation only has to be solved to a relative accuracy well
// above binary32's, since the next binary64 residual measures and corrects
// what the cycle missed; a cycle that cuts eta by less than 10x shows the
// products too coarse for this matrix, and later cycles use binary64 ones --
// except with fp8 factors, whose poor preconditioning is the likelier cause:
// those are refactored in bf16 and keep the binary32 products.
//
// Multi-column blocks are n x nrhs row-major.  Reductions are two-pass with
// fixed order, so results do not depend on scheduling.
#include "common.cuh"
#include "prof.cuh"
#include <cmath>
#include <vector>

namespace lu {

constexpr int kResRows = 32;        // rows per CTA in the residual kernel
constexpr int kResJ = 128;          // columns of A staged per chunk
constexpr int kResRG = 8;           // right-hand sides per register group
constexpr int kRedBlocks = 304;     // partial-sum blocks of the column reductions

// R = B - A X, or R = A X when B is null (the Krylov matvec).  A is n x n (lda), X, B, R are
// n x nrhs (ldx, ldb, ldr).  One CTA: 32 rows x 8 rhs per pass; A's row
// segments stream through registers, X's chunk through shared memory.
__global__ void __launch_bounds__(256) residual_kernel(int n, int nrhs, const double* __restrict__ A, int lda,
                                                       const double* __restrict__ X, int ldx,
                                                       const double* __restrict__ B, int ldb,
                                                       double* __restrict__ R, int ldr) {
    __shared__ double xs[kResJ][kResRG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.x * kResRows + warp * 4;
    for (int g0 = 0; g0 < nrhs; g0 += kResRG) {
        const int ng = min(kResRG, nrhs - g0);
        double acc[4][kResRG];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < kResRG; ++c) acc[r][c] = 0.0;
        for (int j0 = 0; j0 < n; j0 += kResJ) {
            __syncthreads();
            for (int e = threadIdx.x; e < kResJ * kResRG; e += blockDim.x) {
                const int jj = e / kResRG, c = e % kResRG;
                xs[jj][c] = (j0 + jj < n && c < ng) ? X[idx(j0 + jj, g0 + c, ldx)] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = row0 + r;
                if (row >= n) continue;
                const double* arow = A + idx(row, j0, lda);
#pragma unroll
                for (int q = 0; q < kResJ / 32; ++q) {
                    const int jj = lane + 32 * q;
                    const double a = (j0 + jj < n) ? arow[jj] : 0.0;
#pragma unroll
                    for (int c = 0; c < kResRG; ++c) acc[r][c] = fma(a, xs[jj][c], acc[r][c]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < kResRG; ++c) {
                double v = acc[r][c];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                acc[r][c] = v;
            }
        if (lane < kResRG) {
            const int c = lane;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = row0 + r;
                double s = 0.0;
#pragma unroll
                for (int cc = 0; cc < kResRG; ++cc)
                    if (cc == c) s = acc[r][cc];
                if (row < n && c < ng) R[idx(row, g0 + c, ldr)] = B ? B[idx(row, g0 + c, ldb)] - s : s;
            }
        }
    }
}

// W = A Z with binary32 multiplies, for the Krylov products: A's entries and
// Z's are rounded to binary32 and multiplied-added in binary32 over runs of
// kMv32Chunk / 32 terms per lane, each run's sum added into a binary64
// accumulator; the lanes' sums are combined in binary64.  Zf holds one group
// of up to kMv32RG columns of Z in binary32, row-major with stride kMv32RG
// (zf_kernel); A is read once per group.  One warp per kMv32RowsW rows, 16
// warps per CTA.  Zf's chunks of kMv32Chunk rows arrive in shared memory by
// 16-byte asynchronous copies, two buffers so that the next chunk lands
// while the current one is used (row pitch kMv32Pitch: each lane's 16-byte
// reads of its own row hit distinct bank groups).
constexpr int kMv32RG = 16;
constexpr int kMv32RowsW = 2;
constexpr int kMv32Threads = 512;
constexpr int kMv32Rows = (kMv32Threads / 32) * kMv32RowsW;   // rows per CTA
constexpr int kMv32Pitch = kMv32RG + 4;
constexpr int kMv32Chunk = 1024;
constexpr size_t kMv32Smem = 2 * static_cast<size_t>(kMv32Chunk) * kMv32Pitch * sizeof(float);

// Zf[j][c] = (float) Z[j][g0 + c] for c < ng, 0 for ng <= c < kMv32RG.
__global__ void zf_kernel(int n, int g0, int ng, const double* __restrict__ Z, int ldz, float* __restrict__ Zf) {
    const long long tot = static_cast<long long>(n) * kMv32RG;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(e / kMv32RG), c = static_cast<int>(e % kMv32RG);
        Zf[e] = c < ng ? __double2float_rn(Z[idx(j, g0 + c, ldz)]) : 0.f;
    }
}

__global__ void __launch_bounds__(kMv32Threads, 1) matvec32_kernel(int n, int g0, int ng, const double* __restrict__ A,
                                                                   int lda, const float* __restrict__ Zf,
                                                                   double* __restrict__ W, int ldw) {
    extern __shared__ __align__(16) float zs[];         // [2][kMv32Chunk][kMv32Pitch]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.x * kMv32Rows + warp * kMv32RowsW;
    const double* arow[kMv32RowsW];
#pragma unroll
    for (int r = 0; r < kMv32RowsW; ++r) arow[r] = A + idx(min(row0 + r, n - 1), 0, lda);
    const int nchunk = (n + kMv32Chunk - 1) / kMv32Chunk;
    // chunk k -> buffer k & 1: rows j0 .. j0 + nj of Zf, 4 x 16 bytes each
    auto stage = [&](int k) {
        const int j0 = k * kMv32Chunk, nj = min(kMv32Chunk, n - j0);
        float* dst = zs + (k & 1) * kMv32Chunk * kMv32Pitch;
        for (int e = threadIdx.x; e < nj * (kMv32RG / 4); e += kMv32Threads) {
            const int jj = e / (kMv32RG / 4), q = e % (kMv32RG / 4);
            cp_async16(dst + jj * kMv32Pitch + 4 * q, Zf + static_cast<size_t>(j0 + jj) * kMv32RG + 4 * q, 16);
        }
        cp_async_commit();
    };
    double acc[kMv32RowsW][kMv32RG];
#pragma unroll
    for (int r = 0; r < kMv32RowsW; ++r)
#pragma unroll
        for (int c = 0; c < kMv32RG; ++c) acc[r][c] = 0.0;
    stage(0);
    for (int k = 0; k < nchunk; ++k) {
        if (k + 1 < nchunk) {
            stage(k + 1);
            cp_async_wait_1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();                                 // chunk k is in for every thread
        const int j0 = k * kMv32Chunk, nj = min(kMv32Chunk, n - j0);
        const float* zb = zs + (k & 1) * kMv32Chunk * kMv32Pitch;
        float run[kMv32RowsW][kMv32RG];
#pragma unroll
        for (int r = 0; r < kMv32RowsW; ++r)
#pragma unroll
            for (int c = 0; c < kMv32RG; ++c) run[r][c] = 0.f;
#pragma unroll 4
        for (int jj = lane; jj < nj; jj += 32) {
            float a[kMv32RowsW];
#pragma unroll
            for (int r = 0; r < kMv32RowsW; ++r) a[r] = __double2float_rn(arow[r][j0 + jj]);
            const float* zr = zb + jj * kMv32Pitch;
#pragma unroll
            for (int c = 0; c < kMv32RG; c += 4) {
                const float4 z4 = *reinterpret_cast<const float4*>(zr + c);
#pragma unroll
                for (int r = 0; r < kMv32RowsW; ++r) {
                    run[r][c] = fmaf(a[r], z4.x, run[r][c]);
                    run[r][c + 1] = fmaf(a[r], z4.y, run[r][c + 1]);
                    run[r][c + 2] = fmaf(a[r], z4.z, run[r][c + 2]);
                    run[r][c + 3] = fmaf(a[r], z4.w, run[r][c + 3]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kMv32RowsW; ++r)
#pragma unroll
            for (int c = 0; c < kMv32RG; ++c) acc[r][c] += static_cast<double>(run[r][c]);
        __syncthreads();                                 // buffer k & 1 is free for chunk k + 2
    }
#pragma unroll
    for (int r = 0; r < kMv32RowsW; ++r)
#pragma unroll
        for (int c = 0; c < kMv32RG; ++c) {
            double v = acc[r][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            acc[r][c] = v;
        }
    if (lane < kMv32RG) {
        const int c = lane;
#pragma unroll
        for (int r = 0; r < kMv32RowsW; ++r) {
            const int row = row0 + r;
            double v = 0.0;
#pragma unroll
            for (int cc = 0; cc < kMv32RG; ++cc)
                if (cc == c) v = acc[r][cc];
            if (row < n && c < ng) W[idx(row, g0 + c, ldw)] = v;
        }
    }
}

// ||A||_inf: one warp per row, then a max over rows (two-pass).
__global__ void row_abs_sum_kernel(int n, const double* __restrict__ A, int lda, double* __restrict__ part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0;
    for (int r = blockIdx.x * nw + warp; r < n; r += gridDim.x * nw) {
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += fabs(A[idx(r, j, lda)]);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        mx = fmax(mx, s);
    }
    __shared__ double red[32];
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
        part[blockIdx.x] = m;
    }
}

__global__ void max_reduce_kernel(int np, const double* __restrict__ part, double* __restrict__ out) {
    double m = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) m = fmax(m, part[i]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
        *out = r;
    }
}

// Column-wise reductions over an n x nrhs block.  op 0: max |x|; op 1: sum
// x*y (dot); op 2: sum x^2.  Pass 1 writes part[block][c]; pass 2 folds the
// blocks in order.
__global__ void col_reduce_kernel(int n, int nrhs, const double* __restrict__ Xv, int ldx,
                                  const double* __restrict__ Yv, int ldy, int op, double* __restrict__ part) {
    extern __shared__ double sred[];       // blockDim.x
    for (int c = 0; c < nrhs; ++c) {
        double acc = 0.0;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            const double x = Xv[idx(r, c, ldx)];
            if (op == 0) acc = fmax(acc, fabs(x));
            else if (op == 1) acc = fma(x, Yv[idx(r, c, ldy)], acc);
            else acc = fma(x, x, acc);
        }
        sred[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
                sred[threadIdx.x] = (op == 0) ? fmax(sred[threadIdx.x], sred[threadIdx.x + s])
                                              : sred[threadIdx.x] + sred[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[static_cast<size_t>(blockIdx.x) * nrhs + c] = sred[0];
        __syncthreads();
    }
}

__global__ void col_fold_kernel(int nb, int nrhs, int op, const double* __restrict__ part, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double v = part[static_cast<size_t>(b) * nrhs + c];
        acc = (op == 0) ? fmax(acc, v) : acc + v;
    }
    out[c] = acc;
}

// Y (fp32) = X (fp64) * inv_scale[c]   /   X (fp64) = Y (fp32) * scale[c] (+ X when add)
__global__ void to_f32_scaled(int n, int nrhs, const double* __restrict__ X, int ldx, const double* __restrict__ sc,
                              float* __restrict__ Y) {
    const long long tot = static_cast<long long>(n) * nrhs;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
        const double s = sc ? sc[c] : 1.0;
        Y[e] = static_cast<float>(s > 0.0 ? X[idx(r, c, ldx)] / s : 0.0);
    }
}
__global__ void from_f32_scaled(int n, int nrhs, const float* __restrict__ Y, const double* __restrict__ sc,
                                double* __restrict__ X, int ldx, int add) {
    const long long tot = static_cast<long long>(n) * nrhs;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
        const double v = static_cast<double>(Y[e]) * (sc ? sc[c] : 1.0);
        double* p = X + idx(r, c, ldx);
        *p = add ? (*p + v) : v;
    }
}
__global__ void convert_matrix_f32(int n, const double* __restrict__ A, int lda, float* __restrict__ A32) {
    const long long tot = static_cast<long long>(n) * n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / n), c = static_cast<int>(e % n);
        A32[e] = static_cast<float>(A[idx(r, c, lda)]);
    }
}
// Xo[r][c] = sum_i a[i][c] * V_i[r][c]  (+ Xo when add; minus when neg)
__global__ void combine_kernel(int n, int nrhs, int k, const double* __restrict__ V, size_t vstride,
                               const double* __restrict__ coef, double* __restrict__ Xo, int ldx, int add, int neg) {
    const long long tot = static_cast<long long>(n) * nrhs;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(coef[static_cast<size_t>(i) * nrhs + c], V[i * vstride + e], s);
        if (neg) s = -s;
        double* p = Xo + idx(r, c, ldx);
        *p = add ? (*p + s) : s;
    }
}
// H[i][c] = <V_i[:,c], W[:,c]> for i < k: one block per (i, chunk), two-pass.
__global__ void multi_dot_kernel(int n, int nrhs, int k, const double* __restrict__ V, size_t vstride,
                                 const double* __restrict__ W, int nchunk, double* __restrict__ part) {
    extern __shared__ double sred[];
    const int i = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
    const double* Vi = V + i * vstride;
    for (int c = 0; c < nrhs; ++c) {
        double acc = 0.0;
        for (int r = ch * blockDim.x + threadIdx.x; r < n; r += nchunk * blockDim.x)
            acc = fma(Vi[static_cast<size_t>(r) * nrhs + c], W[static_cast<size_t>(r) * nrhs + c], acc);
        sred[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sred[threadIdx.x] += sred[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(static_cast<size_t>(i) * nchunk + ch) * nrhs + c] = sred[0];
        __syncthreads();
    }
}
__global__ void multi_dot_fold(int k, int nrhs, int nchunk, const double* __restrict__ part, double* __restrict__ H) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * nrhs) return;
    const int i = e / nrhs, c = e % nrhs;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[(static_cast<size_t>(i) * nchunk + ch) * nrhs + c];
    H[e] = s;
}

__global__ void eta_kernel(int nr, const double* __restrict__ r, const double* __restrict__ x,
                           const double* __restrict__ b, const double* __restrict__ a, double* __restrict__ o) {
    const int c = threadIdx.x + blockIdx.x * blockDim.x;
    if (c < nr) {
        const double den = a[0] * x[c] + b[c];
        o[c] = den > 0.0 ? r[c] / den : 0.0;
    }
}

// W = R - W and D += W, elementwise over n x nrhs (row-major, stride nrhs).
__global__ void sub_from_kernel(long long tot, const double* __restrict__ R, double* __restrict__ W) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        W[e] = R[e] - W[e];
}
__global__ void add_to_kernel(long long tot, const double* __restrict__ W, double* __restrict__ D) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        D[e] += W[e];
}

static int grid_for(long long tot) {
    long long g = (tot + 255) / 256;
    return static_cast<int>(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// ---------------------------------------------------------------------------
// Host helpers (all stream-ordered)
// ---------------------------------------------------------------------------
struct IrWs {
    double* part = nullptr;   // kRedBlocks * max(nrhs, m+1) * chunks
    double* colv = nullptr;   // nrhs scratch vectors (several)
    double* anorm = nullptr;
    float* r32 = nullptr;     // n x nrhs
};

int residual_f64(int n, int nrhs, const double* A, int lda, const double* X, int ldx, const double* B, int ldb,
                 double* R, int ldr, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    ProfScope ps(LU_PROF_RESIDUAL, s, 2.0 * n * static_cast<double>(n) * nrhs,
                 8.0 * static_cast<double>(n) * n * cdiv(nrhs, kResRG));
    residual_kernel<<<cdiv(n, kResRows), 256, 0, s>>>(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr);
    count_launches(1);
    LU_LAUNCHED();
    return 0;
}

// W = A Z with binary32 multiplies (the Krylov products; see matvec32_kernel).
// zf: scratch of n x kMv32RG floats, 16-byte aligned.
int matvec32(int n, int nrhs, const double* A, int lda, const double* Z, int ldz, double* W, int ldw, float* zf,
             cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    ProfScope ps(LU_PROF_MATVEC32, s, 2.0 * n * static_cast<double>(n) * nrhs,
                 8.0 * static_cast<double>(n) * n * cdiv(nrhs, kMv32RG));
    if (int rc_ = smem_attr(matvec32_kernel, kMv32Smem)) return rc_;
    for (int g0 = 0; g0 < nrhs; g0 += kMv32RG) {
        const int ng = nrhs - g0 < kMv32RG ? nrhs - g0 : kMv32RG;
        zf_kernel<<<grid_for(static_cast<long long>(n) * kMv32RG), 256, 0, s>>>(n, g0, ng, Z, ldz, zf);
        matvec32_kernel<<<cdiv(n, kMv32Rows), kMv32Threads, kMv32Smem, s>>>(n, g0, ng, A, lda, zf, W, ldw);
        count_launches(2);
    }
    LU_LAUNCHED();
    return 0;
}

static int col_reduce(int n, int nrhs, const double* X, int ldx, const double* Y, int ldy, int op, double* part,
                      double* out, cudaStream_t s) {
    ProfScope ps(LU_PROF_RESIDUAL, s);
    col_reduce_kernel<<<kRedBlocks, 256, 256 * sizeof(double), s>>>(n, nrhs, X, ldx, Y, ldy, op, part);
    col_fold_kernel<<<cdiv(nrhs, 64), 64, 0, s>>>(kRedBlocks, nrhs, op, part, out);
    count_launches(2);
    LU_LAUNCHED();
    return 0;
}

int matrix_inf_norm(int n, const double* A, int lda, double* part, double* out, cudaStream_t s) {
    ProfScope ps(LU_PROF_RESIDUAL, s, static_cast<double>(n) * n, 8.0 * static_cast<double>(n) * n);
    row_abs_sum_kernel<<<kRedBlocks, 256, 0, s>>>(n, A, lda, part);
    max_reduce_kernel<<<1, 256, 0, s>>>(kRedBlocks, part, out);
    count_launches(2);
    LU_LAUNCHED();
    return 0;
}

}  // namespace lu

using namespace lu;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int lu_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx, const double* B,
                           int ldb, double* R, int ldr, double* eta, cudaStream_t stream) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && (A == nullptr || lda < n)) return -3;
    if (n > 0 && nrhs > 0 && (X == nullptr || ldx < nrhs)) return -5;
    if (n > 0 && nrhs > 0 && (B == nullptr || ldb < nrhs)) return -7;
    if (n > 0 && nrhs > 0 && eta == nullptr) return -11;
    if (n > 0 && nrhs > 0 && (R == nullptr || ldr < nrhs)) return -9;
    if (n == 0 || nrhs == 0) return 0;
    double* ws = nullptr;
    const size_t words = static_cast<size_t>(kRedBlocks) * nrhs + 4 * static_cast<size_t>(nrhs) + kRedBlocks + 8;
    if (lu_malloc_async(reinterpret_cast<void**>(&ws), words * sizeof(double), stream) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    double* part = ws;
    double* rmax = ws + static_cast<size_t>(kRedBlocks) * nrhs;
    double* xmax = rmax + nrhs;
    double* bmax = xmax + nrhs;
    double* an = bmax + nrhs;
    int rc = residual_f64(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, stream);
    if (!rc) {
        rc = matrix_inf_norm(n, A, lda, part, an, stream);
        if (!rc) rc = col_reduce(n, nrhs, R, ldr, nullptr, 0, 0, part, rmax, stream);
        if (!rc) rc = col_reduce(n, nrhs, X, ldx, nullptr, 0, 0, part, xmax, stream);
        if (!rc) rc = col_reduce(n, nrhs, B, ldb, nullptr, 0, 0, part, bmax, stream);
        if (!rc) {
            eta_kernel<<<cdiv(nrhs, 64), 64, 0, stream>>>(nrhs, rmax, xmax, bmax, an, eta);
            count_launches(1);
            if (cudaPeekAtLastError() != cudaSuccess) {
                cudaGetLastError();
                rc = LU_ELAUNCH;
            }
        }
    }
    cudaFreeAsync(ws, stream);
    return rc;
}

// ---------------------------------------------------------------------------
// ir_solve
// ---------------------------------------------------------------------------
namespace lu {

extern "C" int lu_factor_f32(int m, int n, float* A, int lda, int* piv, int* info, const lu_opts* opts,
                             cudaStream_t stream);

namespace {

struct Dev {
    std::vector<void*> ptrs;
    cudaStream_t s;
    bool ok = true;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        if (lu_malloc_async(&p, count * sizeof(T) + 16, s) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Dev() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

struct IrCtx {
    int n, nrhs;
    const double* A;
    int lda;
    const double* B;
    int ldb;
    double* X;
    int ldx;
    float* A32;       // factors (fp32 storage)
    int* piv;
    const SolvePlan<float>* plan;   // their solve plan
    double* R;        // n x nrhs
    float* r32;       // n x nrhs
    float* zf;        // n x 16: binary32 copy of a Krylov vector (matvec32)
    double* part;     // reduction partials
    double* vec;      // small per-column vectors: [0] scale, [nrhs] eta, ...
    double* an;
    cudaStream_t s;
};

// Z = M^{-1} V (per column: scale by max|v|, fp32 solve, scale back)
int precond_apply(IrCtx& c, const double* V, double* Z, double* scale) {
    if (int rc = col_reduce(c.n, c.nrhs, V, c.nrhs, nullptr, 0, 0, c.part, scale, c.s)) return rc;
    {
        ProfScope ps(LU_PROF_OTHER, c.s);
        to_f32_scaled<<<grid_for(static_cast<long long>(c.n) * c.nrhs), 256, 0, c.s>>>(c.n, c.nrhs, V, c.nrhs, scale,
                                                                                      c.r32);
        count_launches(1);
    }
    LU_LAUNCHED();
    if (int rc = solve_plan_apply<float>(*c.plan, c.nrhs, c.r32, c.nrhs, c.s)) return rc;
    {
        ProfScope ps(LU_PROF_OTHER, c.s);
        from_f32_scaled<<<grid_for(static_cast<long long>(c.n) * c.nrhs), 256, 0, c.s>>>(c.n, c.nrhs, c.r32, scale, Z,
                                                                                        c.nrhs, 0);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

int to_host(cudaStream_t s, const double* d, double* h, int count) {
    LU_TRY(cudaMemcpyAsync(h, d, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    LU_TRY(cudaStreamSynchronize(s));
    return 0;
}

// The correction of one classical step: D = M^{-1} R, then up to J inner
// steps D += M^{-1} (R - A D) with A D in binary32 multiplies, stopping
// before a step whose residual E = R - A D is already within 1e-6 of R
// (the products' accuracy) or did not shrink by 2x in some column.  W is
// scratch (n x nrhs); *steps counts the inner steps applied.
int inner_refine(IrCtx& c, int J, double* D, double* W, int* steps) {
    const int n = c.n, nr = c.nrhs;
    const long long tot = static_cast<long long>(n) * nr;
    double* nrm = c.vec + 6 * nr;
    std::vector<double> rn(nr), prev(nr), en(nr);
    if (int rc = col_reduce(n, nr, c.R, nr, nullptr, 0, 0, c.part, nrm, c.s)) return rc;
    if (int rc = to_host(c.s, nrm, rn.data(), nr)) return rc;
    prev = rn;
    if (int rc = precond_apply(c, c.R, D, c.vec)) return rc;
    for (int j = 0; j < J; ++j) {
        if (int rc = matvec32(n, nr, c.A, c.lda, D, nr, W, nr, c.zf, c.s)) return rc;     // W = A D
        {
            ProfScope ps(LU_PROF_OTHER, c.s);
            sub_from_kernel<<<grid_for(tot), 256, 0, c.s>>>(tot, c.R, W);                  // W = R - A D
            count_launches(1);
        }
        LU_LAUNCHED();
        if (int rc = col_reduce(n, nr, W, nr, nullptr, 0, 0, c.part, nrm, c.s)) return rc;
        if (int rc = to_host(c.s, nrm, en.data(), nr)) return rc;
        bool small = true, shrinks = true;
        for (int k = 0; k < nr; ++k) {
            if (en[k] > 1e-6 * rn[k]) small = false;
            if (en[k] > 0.5 * prev[k]) shrinks = false;
        }
        if (small || !shrinks) break;
        if (int rc = precond_apply(c, W, W, c.vec)) return rc;
        {
            ProfScope ps(LU_PROF_OTHER, c.s);
            add_to_kernel<<<grid_for(tot), 256, 0, c.s>>>(tot, W, D);
            count_launches(1);
        }
        LU_LAUNCHED();
        *steps += 1;
        prev = en;
    }
    return 0;
}

// eta per column of the current X; also leaves R = B - A X.
int backward_error(IrCtx& c, double* eta_h, double* bmax_d) {
    if (int rc = residual_f64(c.n, c.nrhs, c.A, c.lda, c.X, c.ldx, c.B, c.ldb, c.R, c.nrhs, c.s)) return rc;
    double* rmax = c.vec + 2 * c.nrhs;
    double* xmax = c.vec + 3 * c.nrhs;
    double* eta = c.vec + 4 * c.nrhs;
    if (int rc = col_reduce(c.n, c.nrhs, c.R, c.nrhs, nullptr, 0, 0, c.part, rmax, c.s)) return rc;
    if (int rc = col_reduce(c.n, c.nrhs, c.X, c.ldx, nullptr, 0, 0, c.part, xmax, c.s)) return rc;
    eta_kernel<<<cdiv(c.nrhs, 64), 64, 0, c.s>>>(c.nrhs, rmax, xmax, bmax_d, c.an, eta);
    count_launches(1);
    LU_LAUNCHED();
    return to_host(c.s, eta, eta_h, c.nrhs);
}

// One restart cycle of right-preconditioned flexible GMRES on A d = R for
// every column at once; X += d.  Returns the inner iterations done.
int fgmres_cycle(IrCtx& c, int m, double gtol, bool mv32, double* V, double* Z, double* W, double* H,
                 int* iters_out) {
    const int n = c.n, nr = c.nrhs;
    const size_t vs = static_cast<size_t>(n) * nr;
    double* scale = c.vec;
    double* nrm = c.vec + nr;
    std::vector<double> beta(nr), hcol((m + 1) * nr), h2((m + 1) * nr);
    std::vector<double> Hh(static_cast<size_t>(m + 1) * m * nr, 0.0), g(static_cast<size_t>(m + 1) * nr, 0.0);
    std::vector<double> cs(static_cast<size_t>(m) * nr, 0.0), sn(static_cast<size_t>(m) * nr, 0.0);
    // beta = ||R||_2, V0 = R / beta
    if (int rc = col_reduce(n, nr, c.R, nr, nullptr, 0, 2, c.part, nrm, c.s)) return rc;
    if (int rc = to_host(c.s, nrm, beta.data(), nr)) return rc;
    for (int k = 0; k < nr; ++k) {
        beta[k] = std::sqrt(beta[k]);
        g[k] = beta[k];
        hcol[k] = beta[k] > 0.0 ? 1.0 / beta[k] : 0.0;
    }
    LU_TRY(cudaMemcpyAsync(H, hcol.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
    {
        ProfScope ps(LU_PROF_OTHER, c.s);
        combine_kernel<<<grid_for(static_cast<long long>(vs)), 256, 0, c.s>>>(n, nr, 1, c.R, vs, H, V, nr, 0, 0);
        count_launches(1);
    }
    LU_LAUNCHED();
    const int nchunk = 16;
    int j = 0;
    for (; j < m; ++j) {
        double* Vj = V + j * vs;
        double* Zj = Z + j * vs;
        if (int rc = precond_apply(c, Vj, Zj, scale)) return rc;
        if (int rc = mv32 ? matvec32(n, nr, c.A, c.lda, Zj, nr, W, nr, c.zf, c.s)                  // W = A z
                          : residual_f64(n, nr, c.A, c.lda, Zj, nr, nullptr, 0, W, nr, c.s))
            return rc;
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
            {
                ProfScope ps(LU_PROF_OTHER, c.s);
                multi_dot_kernel<<<(j + 1) * nchunk, 256, 256 * sizeof(double), c.s>>>(n, nr, j + 1, V, vs, W,
                                                                                       nchunk, c.part);
                multi_dot_fold<<<cdiv((j + 1) * nr, 128), 128, 0, c.s>>>(j + 1, nr, nchunk, c.part, H);
                combine_kernel<<<grid_for(static_cast<long long>(vs)), 256, 0, c.s>>>(n, nr, j + 1, V, vs, H, W, nr,
                                                                                      1, 1);
                count_launches(3);
            }
            LU_LAUNCHED();
            if (int rc = to_host(c.s, H, pass == 0 ? hcol.data() : h2.data(), (j + 1) * nr)) return rc;
        }
        if (int rc = col_reduce(n, nr, W, nr, nullptr, 0, 2, c.part, nrm, c.s)) return rc;
        std::vector<double> hn(nr);
        if (int rc = to_host(c.s, nrm, hn.data(), nr)) return rc;
        bool all_done = true;
        std::vector<double> inv(nr);
        for (int k = 0; k < nr; ++k) {
            double* Hk = &Hh[static_cast<size_t>(k) * (m + 1) * m];
            for (int i = 0; i <= j; ++i) Hk[i * m + j] = hcol[i * nr + k] + h2[i * nr + k];
            const double hnext = std::sqrt(hn[k]);
            Hk[(j + 1) * m + j] = hnext;
            inv[k] = hnext > 0.0 ? 1.0 / hnext : 0.0;
            // apply earlier rotations, then a new one
            for (int i = 0; i < j; ++i) {
                const double a = Hk[i * m + j], b2 = Hk[(i + 1) * m + j];
                const double cc = cs[i * nr + k], ss = sn[i * nr + k];
                Hk[i * m + j] = cc * a + ss * b2;
                Hk[(i + 1) * m + j] = -ss * a + cc * b2;
            }
            const double a = Hk[j * m + j], b2 = Hk[(j + 1) * m + j];
            const double r = std::hypot(a, b2);
            const double cc = r > 0.0 ? a / r : 1.0, ss = r > 0.0 ? b2 / r : 0.0;
            cs[j * nr + k] = cc;
            sn[j * nr + k] = ss;
            Hk[j * m + j] = r;
            Hk[(j + 1) * m + j] = 0.0;
            const double gj = g[j * nr + k];
            g[j * nr + k] = cc * gj;
            g[(j + 1) * nr + k] = -ss * gj;
            if (std::fabs(g[(j + 1) * nr + k]) > gtol * beta[k] && hnext > 0.0) all_done = false;
        }
        // V_{j+1} = W / h_{j+1}
        LU_TRY(cudaMemcpyAsync(H, inv.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
        {
            ProfScope ps(LU_PROF_OTHER, c.s);
            combine_kernel<<<grid_for(static_cast<long long>(vs)), 256, 0, c.s>>>(n, nr, 1, W, vs, H, V + (j + 1) * vs,
                                                                                  nr, 0, 0);
            count_launches(1);
        }
        LU_LAUNCHED();
        if (all_done) {
            ++j;
            break;
        }
    }
    // y = H^{-1} g (upper triangular j x j), d = Z y, X += d
    std::vector<double> y(static_cast<size_t>(j) * nr, 0.0);
    for (int k = 0; k < nr; ++k) {
        const double* Hk = &Hh[static_cast<size_t>(k) * (m + 1) * m];
        for (int i = j - 1; i >= 0; --i) {
            double t = g[i * nr + k];
            for (int q = i + 1; q < j; ++q) t -= Hk[i * m + q] * y[q * nr + k];
            y[i * nr + k] = Hk[i * m + i] != 0.0 ? t / Hk[i * m + i] : 0.0;
        }
    }
    LU_TRY(cudaMemcpyAsync(H, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, c.s));
    {
        ProfScope ps(LU_PROF_OTHER, c.s);
        combine_kernel<<<grid_for(static_cast<long long>(vs)), 256, 0, c.s>>>(n, nr, j, Z, vs, H, c.X, c.ldx, 1, 0);
        count_launches(1);
    }
    LU_LAUNCHED();
    *iters_out = j;
    return 0;
}

}  // namespace
}  // namespace lu

namespace lu {

// Factor a binary32 copy of A at `prec` (LU_PREC_FP8 / BF16 / F32).
int ir_factor(int n, const double* A, int lda, int prec, int b, int h, IrFactors* f, cudaStream_t s) {
    if (f->A32 == nullptr) {
        if (lu_malloc_async(reinterpret_cast<void**>(&f->A32), static_cast<size_t>(n) * n * sizeof(float) + 16, s) !=
                cudaSuccess ||
            lu_malloc_async(reinterpret_cast<void**>(&f->piv), static_cast<size_t>(n) * sizeof(int) + 16, s) !=
                cudaSuccess ||
            lu_malloc_async(reinterpret_cast<void**>(&f->info), 2 * sizeof(int), s) != cudaSuccess) {
            cudaGetLastError();
            return LU_ENOMEM;
        }
    }
    f->n = n;
    {
        ProfScope ps(LU_PROF_OTHER, s);
        convert_matrix_f32<<<grid_for(static_cast<long long>(n) * n), 256, 0, s>>>(n, A, lda, f->A32);
        count_launches(1);
    }
    LU_LAUNCHED();
    lu_opts fo{};
    fo.b = (prec == LU_PREC_BF16 || prec == LU_PREC_FP8) ? (b + 127) / 128 * 128 : b;
    if (fo.b > 256) fo.b = 256;
    fo.h = h;
    fo.precision = prec;
    f->precision = prec;
    if (int rc = lu_factor_f32(n, n, f->A32, n, f->piv, f->info, &fo, s)) return rc;
    // the solve plan of the new factors (permutation, inverse diagonal blocks)
    solve_plan_free<float>(&f->plan, s);
    return solve_plan_make<float>(n, f->A32, n, f->piv, &f->plan, s);
}

void ir_release(IrFactors* f, cudaStream_t s) {
    solve_plan_free<float>(&f->plan, s);
    if (f->A32) cudaFreeAsync(f->A32, s);
    if (f->piv) cudaFreeAsync(f->piv, s);
    if (f->info) cudaFreeAsync(f->info, s);
    f->A32 = nullptr;
    f->piv = nullptr;
    f->info = nullptr;
}

// Refinement with existing factors (which the ladder may replace by a
// higher-precision factorization).  x0 = M^{-1} B unless keep_x.
int ir_refine(IrFactors* fac, const double* A, int lda, int nrhs, const double* B, int ldb, double* X, int ldx,
              const ir_opts* o, ir_result* res, cudaStream_t stream) {
    const int n = fac->n;
    ir_opts opt{};
    if (o) opt = *o;
    const double tol = opt.tol > 0.0 ? opt.tol : 1e-12;
    const int max_iter = opt.max_iter > 0 ? opt.max_iter : 40;
    const int restart = opt.gmres_restart > 0 ? (opt.gmres_restart < 200 ? opt.gmres_restart : 200) : 30;
    const int b = opt.b > 0 ? opt.b : 128;
    const int h = opt.h > 0 ? opt.h : 128;
    *res = ir_result{};
    res->path = -1;
    res->precision = fac->precision;
    if (n == 0 || nrhs == 0) {
        res->path = 0;
        return 0;
    }
    Dev dev;
    dev.s = stream;
    IrCtx c{};
    c.n = n;
    c.nrhs = nrhs;
    c.A = A;
    c.lda = lda;
    c.B = B;
    c.ldb = ldb;
    c.X = X;
    c.ldx = ldx;
    c.s = stream;
    c.A32 = fac->A32;
    c.piv = fac->piv;
    c.plan = &fac->plan;
    const size_t vs = static_cast<size_t>(n) * nrhs;
    c.R = dev.alloc<double>(vs);
    c.r32 = dev.alloc<float>(vs);
    c.zf = dev.alloc<float>(static_cast<size_t>(n) * kMv32RG);
    const size_t part_words = static_cast<size_t>(kRedBlocks) * nrhs * 4 + static_cast<size_t>(restart + 2) * 16 * nrhs;
    c.part = dev.alloc<double>(part_words);
    c.vec = dev.alloc<double>(8 * static_cast<size_t>(nrhs) + 8);
    c.an = dev.alloc<double>(1);
    double* bmax = dev.alloc<double>(nrhs);
    const int inner = opt.inner_steps < 0 ? 0 : (opt.inner_steps == 0 ? 3 : opt.inner_steps);
    double* Dd = inner > 0 ? dev.alloc<double>(vs) : nullptr;
    double* Wd = inner > 0 ? dev.alloc<double>(vs) : nullptr;
    if (!dev.ok) return LU_ENOMEM;
    double* V = nullptr;
    double* Z = nullptr;
    double* W = nullptr;
    double* H = nullptr;
    if (int rc = matrix_inf_norm(n, A, lda, c.part, c.an, stream)) return rc;
    if (int rc = col_reduce(n, nrhs, B, ldb, nullptr, 0, 0, c.part, bmax, stream)) return rc;
    LU_TRY(cudaMemcpyAsync(&res->info, fac->info, sizeof(int), cudaMemcpyDeviceToHost, stream));
    // x0 = M^{-1} b
    {
        ProfScope ps(LU_PROF_OTHER, stream);
        to_f32_scaled<<<grid_for(static_cast<long long>(vs)), 256, 0, stream>>>(n, nrhs, B, ldb, bmax, c.r32);
        count_launches(1);
    }
    LU_LAUNCHED();
    if (int rc = solve_plan_apply<float>(*c.plan, nrhs, c.r32, nrhs, stream)) return rc;
    {
        ProfScope ps(LU_PROF_OTHER, stream);
        from_f32_scaled<<<grid_for(static_cast<long long>(vs)), 256, 0, stream>>>(n, nrhs, c.r32, bmax, X, ldx, 0);
        count_launches(1);
    }
    LU_LAUNCHED();
    LU_TRY(cudaStreamSynchronize(stream));
    if (res->info < 0) return LU_ETIMEOUT;

    // Precision ladder: the current factorization first; when its refinement
    // stalls, refactor one step up (fp8 -> bf16 -> fp32) and keep refining
    // the current X.
    std::vector<double> eta(nrhs);
    int total_it = 0;
    // Krylov products: binary32 multiplies until a cycle with them gains
    // less than 10x (then binary64 for the rest of the solve)
    bool mv32 = opt.krylov_products != 1;
    for (;;) {
        const bool last = (fac->precision == LU_PREC_F32);
        double prev = 0.0;
        bool krylov = false;
        int cycles = 0;
        bool escalate = false;
        bool last_mv32 = false;      // the cycle just run used binary32 multiplies
        for (;;) {
            if (int rc = backward_error(c, eta.data(), bmax)) return rc;
            double em = 0.0;
            for (double e : eta) em = e > em ? e : em;
            if (total_it == 0 && res->refactors == 0) res->eta0 = em;
            res->eta = em;
            res->iters = total_it;
            res->precision = fac->precision;
            if (em <= tol) {
                res->path = krylov ? 1 : 0;
                return 0;
            }
            if (total_it >= max_iter) return 0;
            // a binary32-product cycle that gained less than 10x: with fp8
            // factors the preconditioner is what failed, so refactor in bf16
            // and keep the binary32 products; otherwise binary64 products from
            // now on.  Either way that cycle does not count below.
            if (last_mv32 && opt.krylov_products == 0 && em > 0.1 * prev) {
                if (fac->precision == LU_PREC_FP8) {
                    escalate = true;
                    break;
                }
                mv32 = false;
                cycles = 0;
            }
            // stall tests: a binary64-product cycle that gains less than 10x,
            // or two of them without reaching tol, move up the ladder
            const bool counted = !last_mv32 || opt.krylov_products == 2;
            if (krylov && counted && !last && (cycles >= 2 || em > 0.1 * prev)) {
                escalate = true;
                break;
            }
            // classical refinement while it contracts by at least 4x per step
            if (!krylov && prev > 0.0 && em > 0.25 * prev) krylov = true;
            prev = em;
            ++total_it;
            if (!krylov) {
                if (inner > 0) {
                    if (int rc = inner_refine(c, inner, Dd, Wd, &res->inner_steps)) return rc;
                    std::swap(c.R, Dd);             // X += D below
                } else if (int rc = precond_apply(c, c.R, c.R, c.vec)) {
                    return rc;
                }
                double* one = c.vec + 5 * nrhs;
                std::vector<double> ones(nrhs, 1.0);
                LU_TRY(cudaMemcpyAsync(one, ones.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, stream));
                {
                    ProfScope ps(LU_PROF_OTHER, stream);
                    combine_kernel<<<grid_for(static_cast<long long>(vs)), 256, 0, stream>>>(n, nrhs, 1, c.R, vs, one,
                                                                                            X, ldx, 1, 0);
                    count_launches(1);
                }
                LU_LAUNCHED();
                LU_TRY(cudaStreamSynchronize(stream));
            } else {
                if (!V) {
                    V = dev.alloc<double>(vs * (restart + 1));
                    Z = dev.alloc<double>(vs * restart);
                    W = dev.alloc<double>(vs);
                    H = dev.alloc<double>(static_cast<size_t>(restart + 1) * nrhs);
                    if (!dev.ok) return LU_ENOMEM;
                }
                int inner = 0;
                // binary32 products: the cycle's inner tolerance stops well above
                // their accuracy; binary64: the usual 1e-10
                if (int rc = fgmres_cycle(c, restart, mv32 ? 1e-6 : 1e-10, mv32, V, Z, W, H, &inner)) return rc;
                res->gmres_iters += inner;
                last_mv32 = mv32;
                if (mv32)
                    res->cycles32 += 1;
                else
                    res->cycles64 += 1;
                if (!mv32 || opt.krylov_products == 2) ++cycles;
            }
        }
        if (!escalate) return 0;
        const int up = (fac->precision == LU_PREC_FP8) ? LU_PREC_BF16 : LU_PREC_F32;
        if (int rc = ir_factor(n, A, lda, up, b, h, fac, stream)) return rc;
        res->refactors += 1;
        LU_TRY(cudaMemcpyAsync(&res->info, fac->info, sizeof(int), cudaMemcpyDeviceToHost, stream));
        LU_TRY(cudaStreamSynchronize(stream));
        if (res->info < 0) return LU_ETIMEOUT;
    }
}

size_t ir_workspace_bytes(int n, int nrhs, int restart) {
    const size_t vs = static_cast<size_t>(n) * nrhs;
    if (restart <= 0) restart = 30;
    return vs * (8 + 4 + 8 * (2 * static_cast<size_t>(restart) + 2) + 16) + static_cast<size_t>(n) * kMv32RG * 4 +
           (static_cast<size_t>(kRedBlocks) * nrhs * 4 + static_cast<size_t>(restart + 2) * 16 * nrhs + 16 * nrhs) * 8 +
           4096;
}

}  // namespace lu

extern "C" int ir_solve(int n, int nrhs, const double* A, int lda, const double* B, int ldb, double* X, int ldx,
                        const ir_opts* o, ir_result* res, cudaStream_t stream) {
    using namespace lu;
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > 384) return -2;
    if (n > 0 && (A == nullptr || lda < n)) return -3;
    if (n > 0 && nrhs > 0 && (B == nullptr || ldb < nrhs)) return -5;
    if (n > 0 && nrhs > 0 && (X == nullptr || ldx < nrhs)) return -7;
    if (res == nullptr) return -10;
    ir_opts opt{};
    if (o) opt = *o;
    const int prec = opt.precision ? opt.precision : LU_PREC_BF16;
    if (prec < LU_PREC_F64 || prec > LU_PREC_FP8) return -9;
    if (opt.krylov_products < 0 || opt.krylov_products > 2) return -11;
    *res = ir_result{};
    res->path = -1;
    if (n == 0 || nrhs == 0) {
        res->path = 0;
        return 0;
    }
    IrFactors fac{};
    const int b = opt.b > 0 ? opt.b : 128;
    const int h = opt.h > 0 ? opt.h : 128;
    int rc = ir_factor(n, A, lda, prec == LU_PREC_F64 ? LU_PREC_F32 : prec, b, h, &fac, stream);
    if (!rc) rc = ir_refine(&fac, A, lda, nrhs, B, ldb, X, ldx, &opt, res, stream);
    ir_release(&fac, stream);
    return rc;
}

// ---------------------------------------------------------------------------
// lu_residual_noalloc: lu_residual for callers that cannot allocate device
// memory while they run -- for example a serving loop that reserves all of
// its memory up front so that no request can fail halfway on an allocation,
// or a process whose GPU memory is owned by another framework's caching
// allocator.  Its reduction scratch is a fixed array in this file instead of
// a pool buffer, which bounds nrhs.
// ---------------------------------------------------------------------------
namespace lu {

constexpr int kNoAllocMaxRhs = 64;
constexpr size_t kNoAllocWords =
    static_cast<size_t>(kRedBlocks) * kNoAllocMaxRhs + 4 * static_cast<size_t>(kNoAllocMaxRhs) + kRedBlocks + 8;

// Shared by every call on a device, held until the process exits (about
// 160 KB per device that loads the library).  Every slot a call reads is
// written earlier in the same call, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];

namespace {
// Device address of this device's scratch array.  In host code the array's
// name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call (a cheap host-side query): an address kept from an earlier call would
// point into a destroyed context after cudaDeviceReset.
int noalloc_scratch(double** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return LU_ELAUNCH;
    }
    *out = static_cast<double*>(p);
    return 0;
}
}  // namespace
}  // namespace lu

extern "C" int lu_residual_noalloc(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                                   const double* B, int ldb, double* R, int ldr, double* eta, cudaStream_t stream) {
    using namespace lu;
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > kNoAllocMaxRhs) return -2;
    if (n > 0 && (A == nullptr || lda < n)) return -3;
    if (n > 0 && nrhs > 0 && (X == nullptr || ldx < nrhs)) return -5;
    if (n > 0 && nrhs > 0 && (B == nullptr || ldb < nrhs)) return -7;
    if (n > 0 && nrhs > 0 && (R == nullptr || ldr < nrhs)) return -9;
    if (n > 0 && nrhs > 0 && eta == nullptr) return -11;
    if (n == 0 || nrhs == 0) return 0;
    double* ws = nullptr;
    if (int rc = noalloc_scratch(&ws)) return rc;
    double* part = ws;
    double* rmax = ws + static_cast<size_t>(kRedBlocks) * kNoAllocMaxRhs;
    double* xmax = rmax + kNoAllocMaxRhs;
    double* bmax = xmax + kNoAllocMaxRhs;
    double* an = bmax + kNoAllocMaxRhs;
    residual_kernel<<<cdiv(n, kResRows), 256, 0, stream>>>(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr);
    row_abs_sum_kernel<<<kRedBlocks, 256, 0, stream>>>(n, A, lda, part);
    max_reduce_kernel<<<1, 256, 0, stream>>>(kRedBlocks, part, an);
    col_reduce_kernel<<<kRedBlocks, 256, 256 * sizeof(double), stream>>>(n, nrhs, R, ldr, nullptr, 0, 0, part);
    col_fold_kernel<<<cdiv(nrhs, 64), 64, 0, stream>>>(kRedBlocks, nrhs, 0, part, rmax);
    col_reduce_kernel<<<kRedBlocks, 256, 256 * sizeof(double), stream>>>(n, nrhs, X, ldx, nullptr, 0, 0, part);
    col_fold_kernel<<<cdiv(nrhs, 64), 64, 0, stream>>>(kRedBlocks, nrhs, 0, part, xmax);
    col_reduce_kernel<<<kRedBlocks, 256, 256 * sizeof(double), stream>>>(n, nrhs, B, ldb, nullptr, 0, 0, part);
    col_fold_kernel<<<cdiv(nrhs, 64), 64, 0, stream>>>(kRedBlocks, nrhs, 0, part, bmax);
    eta_kernel<<<cdiv(nrhs, 64), 64, 0, stream>>>(nrhs, rmax, xmax, bmax, an, eta);
    count_launches(10);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return LU_ELAUNCH;
    }
    return 0;
}
