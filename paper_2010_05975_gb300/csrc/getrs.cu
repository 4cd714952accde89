// Solve A X = B with the factors P A = L U (getrs): X = U^{-1} L^{-1} P B.
// The linear solve is what the paper's factorization serves ("linear
// solvers", Section 1); the paper does not spell it out.
//
// 1. The swap sequence piv is composed into one permutation (one thread,
//    in shared memory when it fits) and B is gathered into a workspace Y.
// 2. Forward substitution with unit L, then back substitution with U, both
//    blocked by NB rows with inverted diagonal blocks (below).
// 3. The result is copied back into B.
#include "common.cuh"
#include "prof.cuh"

namespace lu {

constexpr int kPermSmemMax = 49152;     // ints held in shared memory

__global__ void perm_from_piv_smem(int n, const int* __restrict__ piv, int* __restrict__ perm) {
    extern __shared__ int sp[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sp[i] = i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < n; ++i) {
            const int p = piv[i];
            const int t = sp[i];
            sp[i] = sp[p];
            sp[p] = t;
        }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = sp[i];
}

__global__ void perm_from_piv_global(int n, const int* __restrict__ piv, int* __restrict__ perm) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < n; ++i) {
            const int p = piv[i];
            const int t = perm[i];
            perm[i] = perm[p];
            perm[p] = t;
        }
}

template <typename T>
__global__ void gather_rows(int n, int nrhs, const int* __restrict__ perm, const T* __restrict__ B, int ldb,
                            T* __restrict__ Y) {
    const long long tot = static_cast<long long>(n) * nrhs;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
        Y[e] = B[idx(perm[i], c, ldb)];
    }
}

template <typename T>
__global__ void copy_out(int n, int nrhs, const T* __restrict__ Y, T* __restrict__ B, int ldb) {
    const long long tot = static_cast<long long>(n) * nrhs;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
        B[idx(i, c, ldb)] = Y[e];
    }
}

// Blocked solves use the inverses of the diagonal blocks: one launch inverts
// every NB x NB diagonal block of L (unit lower) and U (upper); each block
// step is then  X_I = inv(D_I) Y_I  (a small product, several CTAs)  and
// Y_J -= T_{J,I} X_I  for the rows that remain (grid-wide).  NB = 128 for
// binary32, 64 for binary64 (two NB x NB tiles fit in shared memory).
template <typename T>
struct SolveNB {
    static constexpr int value = sizeof(T) == 4 ? 128 : 64;
};

// One CTA per (block, factor): Dinv[blk][kind] = inv(diag block).  Thread c
// owns column c of the inverse; the block stays in shared memory.
template <typename T>
__global__ void __launch_bounds__(128) invert_diag_kernel(int n, const T* __restrict__ LU, int lda,
                                                          T* __restrict__ Dinv) {
    constexpr int NB = SolveNB<T>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);              // NB x (NB+1)
    T* Xs = S + NB * (NB + 1);                           // NB x (NB+1), column c at Xs[p][c]
    const int blk = blockIdx.x, kind = blockIdx.y;       // 0: L (unit lower), 1: U (upper)
    const int r0 = blk * NB, nb = min(NB, n - r0);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        S[i * (NB + 1) + j] = (i < nb && j < nb) ? LU[idx(r0 + i, r0 + j, lda)] : T(0);
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < NB) {
        if (kind == 0) {
            for (int i = 0; i < NB; ++i) {
                T s = (i == c) ? T(1) : T(0);
                if (i > c && i < nb) {
                    for (int p = c; p < i; ++p) s = fma(-S[i * (NB + 1) + p], Xs[p * (NB + 1) + c], s);
                }
                Xs[i * (NB + 1) + c] = (i < nb && c < nb) ? s : T(0);
            }
        } else {
            for (int i = NB - 1; i >= 0; --i) {
                T s = (i == c) ? T(1) : T(0);
                if (i <= c && c < nb) {
                    for (int p = i + 1; p <= c; ++p) s = fma(-S[i * (NB + 1) + p], Xs[p * (NB + 1) + c], s);
                    s = s / S[i * (NB + 1) + i];
                } else {
                    s = T(0);
                }
                Xs[i * (NB + 1) + c] = s;
            }
        }
    }
    __syncthreads();
    T* out = Dinv + (static_cast<size_t>(blk) * 2 + kind) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = Xs[(e / NB) * (NB + 1) + (e % NB)];
}

// X[r0+i][:] = sum_p D[i][p] Y[r0+p][:] for the rows this CTA owns (16 per CTA).
template <typename T>
__global__ void __launch_bounds__(256) diag_apply_kernel(int nrhs, int r0, int nb, const T* __restrict__ D,
                                                         const T* __restrict__ Y, T* __restrict__ X) {
    constexpr int NB = SolveNB<T>::value;
    const int i0 = blockIdx.x * 16;
    const int tot = 16 * nrhs;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int i = i0 + e / nrhs, c = e % nrhs;
        if (i >= nb) continue;
        T s = 0;
        for (int p = 0; p < nb; ++p) s = fma(D[i * NB + p], Y[idx(r0 + p, c, nrhs)], s);
        X[idx(r0 + i, c, nrhs)] = s;
    }
}

// Y[r][:] -= LU[r][r0:r0+nb] * X[r0:r0+nb][:] for r in [ra, rb).
// nrhs >= 8: one thread per (row, column); else one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) block_update(int nrhs, int ra, int rb, int r0, int nb,
                                                    const T* __restrict__ LU, int lda, const T* __restrict__ X,
                                                    T* __restrict__ Y) {
    constexpr int NB = SolveNB<T>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Xs = reinterpret_cast<T*>(smem_raw);          // nb x nrhs
    for (int e = threadIdx.x; e < nb * nrhs; e += blockDim.x) Xs[e] = X[static_cast<size_t>(r0) * nrhs + e];
    __syncthreads();
    if (nrhs >= 8) {
        const long long pairs = static_cast<long long>(rb - ra) * nrhs;
        for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < pairs;
             e += static_cast<long long>(gridDim.x) * blockDim.x) {
            const int r = ra + static_cast<int>(e / nrhs), c = static_cast<int>(e % nrhs);
            const T* lrow = LU + idx(r, r0, lda);
            T s = 0;
            for (int p = 0; p < nb; ++p) s = fma(lrow[p], Xs[p * nrhs + c], s);
            Y[idx(r, c, nrhs)] -= s;
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = ra + blockIdx.x * nwarp + warp; r < rb; r += gridDim.x * nwarp) {
        const T* lrow = LU + idx(r, r0, lda);
        T lv[NB / 32];
#pragma unroll
        for (int e = 0; e < NB / 32; ++e) {
            const int p = lane + 32 * e;
            lv[e] = p < nb ? lrow[p] : T(0);
        }
        for (int c = 0; c < nrhs; ++c) {
            T s = 0;
#pragma unroll
            for (int e = 0; e < NB / 32; ++e) {
                const int p = lane + 32 * e;
                if (p < nb) s = fma(lv[e], Xs[p * nrhs + c], s);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) Y[idx(r, c, nrhs)] -= s;
        }
    }
}

template <typename T>
int getrs_impl(int n, int nrhs, const T* LU, int lda, const int* piv, T* B, int ldb, int* perm, T* Y, T* X,
               T* Dinv, cudaStream_t s) {
    constexpr int NB = SolveNB<T>::value;
    if (n <= kPermSmemMax) {
        const size_t smem = static_cast<size_t>(n) * sizeof(int);
        if (int rc_ = smem_attr(perm_from_piv_smem, smem)) return rc_;
        ProfScope ps(LU_PROF_SOLVE, s);
        perm_from_piv_smem<<<1, 256, smem, s>>>(n, piv, perm);
        count_launches(1);
    } else {
        ProfScope ps(LU_PROF_SOLVE, s);
        perm_from_piv_global<<<1, 256, 0, s>>>(n, piv, perm);
        count_launches(1);
    }
    LU_LAUNCHED();
    const long long tot = static_cast<long long>(n) * nrhs;
    const int gblocks = static_cast<int>(tot / 256 + 1 < 4096 ? tot / 256 + 1 : 4096);
    const int nblk = cdiv(n, NB);
    {
        ProfScope ps(LU_PROF_SOLVE, s);
        gather_rows<T><<<gblocks, 256, 0, s>>>(n, nrhs, perm, B, ldb, Y);
        count_launches(1);
    }
    LU_LAUNCHED();
    {
        const size_t ismem = 2 * static_cast<size_t>(NB) * (NB + 1) * sizeof(T);
        if (int rc_ = smem_attr(invert_diag_kernel<T>, ismem)) return rc_;
        ProfScope ps(LU_PROF_SOLVE, s);
        invert_diag_kernel<T><<<dim3(nblk, 2), 128, ismem, s>>>(n, LU, lda, Dinv);
        count_launches(1);
    }
    LU_LAUNCHED();
    const size_t usmem = static_cast<size_t>(NB) * nrhs * sizeof(T);
    if (int rc_ = smem_attr(block_update<T>, usmem)) return rc_;
    auto update_grid = [&](int rows) {
        const long long work = (nrhs >= 8) ? static_cast<long long>(rows) * nrhs : static_cast<long long>(rows) * 32;
        const long long g = (work + 255) / 256;
        return static_cast<int>(g < 2048 ? (g > 0 ? g : 1) : 2048);
    };
    // forward: Y (= P B) -> X = L^{-1} P B
    for (int bi = 0; bi < nblk; ++bi) {
        const int r0 = bi * NB, nb = min(NB, n - r0);
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            diag_apply_kernel<T><<<cdiv(nb, 16), 256, 0, s>>>(nrhs, r0, nb, Dinv + static_cast<size_t>(bi) * 2 * NB * NB,
                                                              Y, X);
            count_launches(1);
        }
        LU_LAUNCHED();
        const int rows = n - (r0 + nb);
        if (rows > 0) {
            ProfScope ps(LU_PROF_SOLVE, s, 2.0 * rows * nb * nrhs);
            block_update<T><<<update_grid(rows), 256, usmem, s>>>(nrhs, r0 + nb, n, r0, nb, LU, lda, X, Y);
            count_launches(1);
        }
        LU_LAUNCHED();
    }
    // backward: the forward result X becomes the right-hand side; Y receives U^{-1} X
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int r0 = bi * NB, nb = min(NB, n - r0);
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            diag_apply_kernel<T><<<cdiv(nb, 16), 256, 0, s>>>(
                nrhs, r0, nb, Dinv + (static_cast<size_t>(bi) * 2 + 1) * NB * NB, X, Y);
            count_launches(1);
        }
        LU_LAUNCHED();
        if (r0 > 0) {
            ProfScope ps(LU_PROF_SOLVE, s, 2.0 * r0 * nb * nrhs);
            block_update<T><<<update_grid(r0), 256, usmem, s>>>(nrhs, 0, r0, r0, nb, LU, lda, Y, X);
            count_launches(1);
        }
        LU_LAUNCHED();
    }
    {
        ProfScope ps(LU_PROF_SOLVE, s);
        copy_out<T><<<gblocks, 256, 0, s>>>(n, nrhs, Y, B, ldb);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template <typename T>
int getrs_alloc(int n, int nrhs, const T* LU, int lda, const int* piv, T* B, int ldb, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    constexpr int NB = SolveNB<T>::value;
    const size_t vs = static_cast<size_t>(n) * nrhs;
    const size_t dsz = static_cast<size_t>(cdiv(n, NB)) * 2 * NB * NB;
    void* ws = nullptr;
    const size_t bytes = sizeof(int) * static_cast<size_t>(n) + 64 + sizeof(T) * (2 * vs + dsz) + 64;
    if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    int* perm = static_cast<int*>(ws);
    T* Y = reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(perm + n + 16) & ~uintptr_t(15));
    T* X = Y + vs;
    T* Dinv = X + vs;
    int rc = getrs_impl<T>(n, nrhs, LU, lda, piv, B, ldb, perm, Y, X, Dinv, s);
    cudaFreeAsync(ws, s);
    return rc;
}

int getrs_f64(int n, int nrhs, const double* LU, int lda, const int* piv, double* B, int ldb, cudaStream_t s) {
    return getrs_alloc<double>(n, nrhs, LU, lda, piv, B, ldb, s);
}

int getrs_f32(int n, int nrhs, const float* LU, int lda, const int* piv, float* B, int ldb, cudaStream_t s) {
    return getrs_alloc<float>(n, nrhs, LU, lda, piv, B, ldb, s);
}

}  // namespace lu
