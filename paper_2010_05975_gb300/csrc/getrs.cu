// Solve A X = B with the factors P A = L U (getrs): X = U^{-1} L^{-1} P B.
// The linear solve is what the paper's factorization serves ("linear
// solvers", Section 1); the paper does not spell it out.
//
// 1. The swap sequence piv is composed into one permutation (one thread,
//    in shared memory when it fits) and B is gathered into a workspace Y.
// 2. Forward substitution with unit L, then back substitution with U, both
//    blocked by NB rows: a one-CTA kernel solves the diagonal block, and a
//    grid-wide kernel subtracts that block's contribution from the rows that
//    remain.
// 3. Y is copied back into B.
#include "common.cuh"
#include "prof.cuh"

namespace lu {

constexpr int kSolveNB = 64;
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

// Diagonal block rows [r0, r0+nb): forward (unit lower) or backward (upper,
// divide by the diagonal).  One thread per right-hand side column.
template <typename T, bool kLower>
__global__ void diag_solve(int nrhs, int r0, int nb, const T* __restrict__ LU, int lda, T* __restrict__ Y) {
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        if (kLower) {
            for (int i = 1; i < nb; ++i) {
                T s = Y[idx(r0 + i, c, nrhs)];
                for (int p = 0; p < i; ++p) s = fma(-LU[idx(r0 + i, r0 + p, lda)], Y[idx(r0 + p, c, nrhs)], s);
                Y[idx(r0 + i, c, nrhs)] = s;
            }
        } else {
            for (int i = nb - 1; i >= 0; --i) {
                T s = Y[idx(r0 + i, c, nrhs)];
                for (int p = i + 1; p < nb; ++p) s = fma(-LU[idx(r0 + i, r0 + p, lda)], Y[idx(r0 + p, c, nrhs)], s);
                Y[idx(r0 + i, c, nrhs)] = s / LU[idx(r0 + i, r0 + i, lda)];
            }
        }
    }
}

// Y[r, :] -= LU[r, r0:r0+nb] * Y[r0:r0+nb, :] for r in [ra, rb).  A warp per
// row; lanes split the nb terms and reduce with shuffles per column.
template <typename T>
__global__ void __launch_bounds__(256) block_update(int nrhs, int ra, int rb, int r0, int nb,
                                                    const T* __restrict__ LU, int lda, T* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ys = reinterpret_cast<T*>(smem_raw);          // nb x nrhs
    for (int e = threadIdx.x; e < nb * nrhs; e += blockDim.x) Ys[e] = Y[static_cast<size_t>(r0) * nrhs + e];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = ra + blockIdx.x * nwarp + warp; r < rb; r += gridDim.x * nwarp) {
        const T* lrow = LU + idx(r, r0, lda);
        T lv[kSolveNB / 32];
#pragma unroll
        for (int e = 0; e < kSolveNB / 32; ++e) {
            const int p = lane + 32 * e;
            lv[e] = p < nb ? lrow[p] : T(0);
        }
        for (int c = 0; c < nrhs; ++c) {
            T s = 0;
#pragma unroll
            for (int e = 0; e < kSolveNB / 32; ++e) {
                const int p = lane + 32 * e;
                if (p < nb) s = fma(lv[e], Ys[p * nrhs + c], s);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) Y[idx(r, c, nrhs)] -= s;
        }
    }
}

template <typename T>
int getrs_impl(int n, int nrhs, const T* LU, int lda, const int* piv, T* B, int ldb, int* perm, T* Y,
               cudaStream_t s) {
    if (n <= kPermSmemMax) {
        const size_t smem = static_cast<size_t>(n) * sizeof(int);
        LU_TRY(cudaFuncSetAttribute(perm_from_piv_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            perm_from_piv_smem<<<1, 256, smem, s>>>(n, piv, perm);
            count_launches(1);
        }
    } else {
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            perm_from_piv_global<<<1, 256, 0, s>>>(n, piv, perm);
            count_launches(1);
        }
    }
    LU_LAUNCHED();
    const long long tot = static_cast<long long>(n) * nrhs;
    const int gblocks = static_cast<int>(tot / 256 + 1 < 4096 ? tot / 256 + 1 : 4096);
    {
        ProfScope ps(LU_PROF_SOLVE, s);
        gather_rows<T><<<gblocks, 256, 0, s>>>(n, nrhs, perm, B, ldb, Y);
        count_launches(1);
    }
    LU_LAUNCHED();
    const size_t usmem = static_cast<size_t>(kSolveNB) * nrhs * sizeof(T);
    LU_TRY(cudaFuncSetAttribute(block_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(usmem)));
    for (int r0 = 0; r0 < n; r0 += kSolveNB) {
        const int nb = min(kSolveNB, n - r0);
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            diag_solve<T, true><<<1, 64, 0, s>>>(nrhs, r0, nb, LU, lda, Y);
            count_launches(1);
        }
        LU_LAUNCHED();
        const int rows = n - (r0 + nb);
        if (rows > 0) {
            const int blocks = min(cdiv(rows, 8), 2 * 152);
            {
                ProfScope ps(LU_PROF_SOLVE, s);
                block_update<T><<<blocks, 256, usmem, s>>>(nrhs, r0 + nb, n, r0, nb, LU, lda, Y);
                count_launches(1);
            }
            LU_LAUNCHED();
        }
    }
    const int nblk = cdiv(n, kSolveNB);
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int r0 = bi * kSolveNB;
        const int nb = min(kSolveNB, n - r0);
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            diag_solve<T, false><<<1, 64, 0, s>>>(nrhs, r0, nb, LU, lda, Y);
            count_launches(1);
        }
        LU_LAUNCHED();
        if (r0 > 0) {
            const int blocks = min(cdiv(r0, 8), 2 * 152);
            {
                ProfScope ps(LU_PROF_SOLVE, s);
                block_update<T><<<blocks, 256, usmem, s>>>(nrhs, 0, r0, r0, nb, LU, lda, Y);
                count_launches(1);
            }
            LU_LAUNCHED();
        }
    }
    {
        ProfScope ps(LU_PROF_SOLVE, s);
        copy_out<T><<<gblocks, 256, 0, s>>>(n, nrhs, Y, B, ldb);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

int getrs_f64(int n, int nrhs, const double* LU, int lda, const int* piv, double* B, int ldb, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    int* perm = nullptr;
    double* Y = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&perm), sizeof(int) * static_cast<size_t>(n), s) != cudaSuccess)
        return LU_ENOMEM;
    if (cudaMallocAsync(reinterpret_cast<void**>(&Y), sizeof(double) * static_cast<size_t>(n) * nrhs, s) !=
        cudaSuccess) {
        cudaFreeAsync(perm, s);
        return LU_ENOMEM;
    }
    int rc = getrs_impl<double>(n, nrhs, LU, lda, piv, B, ldb, perm, Y, s);
    cudaFreeAsync(Y, s);
    cudaFreeAsync(perm, s);
    return rc;
}

}  // namespace lu

namespace lu {
int getrs_f32(int n, int nrhs, const float* LU, int lda, const int* piv, float* B, int ldb, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    int* perm = nullptr;
    float* Y = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&perm), sizeof(int) * static_cast<size_t>(n), s) != cudaSuccess)
        return LU_ENOMEM;
    if (cudaMallocAsync(reinterpret_cast<void**>(&Y), sizeof(float) * static_cast<size_t>(n) * nrhs, s) !=
        cudaSuccess) {
        cudaFreeAsync(perm, s);
        return LU_ENOMEM;
    }
    int rc = getrs_impl<float>(n, nrhs, LU, lda, piv, B, ldb, perm, Y, s);
    cudaFreeAsync(Y, s);
    cudaFreeAsync(perm, s);
    return rc;
}
}  // namespace lu
