// Solve A X = B with the factors P A = L U (getrs): X = U^{-1} L^{-1} P B.
// The linear solve is what the paper's factorization serves ("linear
// solvers", Section 1); the paper does not spell it out.  A Cholesky factor
// L goes through the same machinery with U = L^T and no permutation.
//
// A solve plan holds what depends on the factors only: the row permutation
// composed from the swap sequence piv, and the inverses of the NB x NB
// diagonal blocks of L (unit lower) and U (upper), stored transposed.  The
// refinement keeps one plan per factorization; the one-shot entry points
// build and drop one per call.
//
// Applying a plan: B is gathered through the permutation into Y (row stride
// nc, padded to a width of 8, 16, 32 or 64), then one kernel runs the
// blocked forward and backward substitutions as a list of work items taken
// in order from an atomic counter.  Every item is a 32-row contraction:
//   forward step b:   parts of X_b = inv(L_bb) Y_b (32 rows each), then for
//                     every 32-row tile t below the block: Y_t -= L_tb X_b;
//   backward step b:  (b from the last block up) the parts of
//                     X_b = inv(U_bb) X_b, then the tiles above:
//                     X_t -= U_tb X_b.
// An item first stages its coefficient rows, then waits (bounded, through
// per-tile and per-block counters) on items earlier in the list, which CTAs
// already running have taken, so the kernel progresses whatever number of
// its CTAs is resident.  Each tile takes its updates one step at a time, in
// step order, so results do not depend on timing.  Right-hand sides go
// through in passes of up to 64.
#include "common.cuh"
#include "prof.cuh"
#include <mutex>

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

// Block size of the substitution: NB = 128 for binary32, 64 for binary64
// (the inversion kernel holds two NB x NB tiles in shared memory).
template <typename T>
struct SolveNB {
    static constexpr int value = sizeof(T) == 4 ? 128 : 64;
};

// One CTA per (block, factor): Dinv[blk][kind] = inv(diag block).  Thread c
// owns column c of the inverse; the block stays in shared memory.  With
// chol set the factors are L (non-unit lower, from a Cholesky factorization)
// and L^T: both kinds compute inv(L_bb), kind 1 stores inv(L_bb^T) =
// inv(L_bb)^T.
template <typename T>
__global__ void __launch_bounds__(128) invert_diag_kernel(int n, const T* __restrict__ LU, int lda,
                                                          T* __restrict__ Dinv, int chol) {
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
        if (chol) {
            for (int i = 0; i < NB; ++i) {
                T s = (i == c) ? T(1) : T(0);
                if (i >= c && i < nb && c < nb) {
                    for (int p = c; p < i; ++p) s = fma(-S[i * (NB + 1) + p], Xs[p * (NB + 1) + c], s);
                    s = s / S[i * (NB + 1) + i];
                } else {
                    s = T(0);
                }
                Xs[i * (NB + 1) + c] = s;
            }
        } else if (kind == 0) {
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
    // transposed: out[p][i] = inv[i][p], so that a warp reads consecutive i
    T* out = Dinv + (static_cast<size_t>(blk) * 2 + kind) * NB * NB;
    if (chol && kind == 1) {
        // out[p][i] = inv(L^T)[i][p] = inv(L)[p][i]
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = Xs[(e / NB) * (NB + 1) + (e % NB)];
    } else {
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = Xs[(e % NB) * (NB + 1) + (e / NB)];
    }
}

constexpr int kSolveRhs = 64;            // right-hand sides per pass
constexpr int kSolveTile = 32;           // rows per update tile
constexpr int kSolveThreads = 256;

// Item list bookkeeping (device memory, zeroed before each pass).
struct SolveSync {
    int next;          // next item to take
    int timeout;
    int pad[2];
};

// Items before forward step b / backward step b: off[0..2*nblk], built once
// per plan (the block size arrives in off[0]).
__global__ void solve_offsets_kernel(int n, int* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    constexpr int TR = kSolveTile;
    const int ntile = cdiv(n, TR);
    const int NB = off[0];
    const int nblk = cdiv(n, NB);
    const int tpb = NB / TR;
    int acc = 0;
    for (int b = 0; b < nblk; ++b) {                    // forward
        off[b] = acc;
        const int parts = cdiv(min(NB, n - b * NB), TR);
        acc += parts + ntile - min(ntile, (b + 1) * tpb);
    }
    for (int st = 0; st < nblk; ++st) {                 // backward, last block first
        const int b = nblk - 1 - st;
        off[nblk + st] = acc;
        const int parts = cdiv(min(NB, n - b * NB), TR);
        acc += parts + b * tpb;
    }
    off[2 * nblk] = acc;
}

// Wait by thread 0 until *flag >= want, at most limit_ns of wall-clock time
// (%globaltimer, read every 64 polls); a wait that runs out records the
// timeout.  After any timeout every wait returns at once, so a broken run
// ends quickly (its results are then invalid and the host reports
// LU_ETIMEOUT).
__device__ __forceinline__ void solve_wait(const int* flag, int want, SolveSync* sy, unsigned long long limit_ns) {
    const volatile int* f = flag;
    const volatile int* to = &sy->timeout;
    unsigned long long t0 = 0;
    for (unsigned it = 1; *f < want; ++it) {
        if ((it & 63) == 0) {
            if (*to) return;
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                atomicExch(&sy->timeout, 1);
                return;
            }
        }
        __nanosleep(32);
    }
}

// Forward (L: Y -> X) then backward (U: X -> Y) substitution; right-hand
// sides row-major with stride NCW (columns >= nc are zero and stay zero).
// With chol set, U is L^T: the backward tiles read L transposed.
template <typename T, int NCW>
__global__ void __launch_bounds__(kSolveThreads) solve_items_kernel(int n, const T* __restrict__ LU, int lda,
                                                                    const T* __restrict__ DT,
                                                                    const int* __restrict__ off, T* Y, T* X,
                                                                    int* fdone, int* bdone, int* xpf, int* xpb,
                                                                    SolveSync* sy, int chol,
                                                                    unsigned long long wait_ns, int inject) {
    constexpr int NB = SolveNB<T>::value;
    constexpr int TR = kSolveTile;
    constexpr int TPB = NB / TR;                     // tiles (and solve parts) per block
    constexpr int MU = NCW / 8;                      // columns per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ls = reinterpret_cast<T*>(smem_raw);          // TR x (NB+1): the item's coefficient rows
    T* Bs = Ls + TR * (NB + 1);                      // NB x NCW: the right operand
    __shared__ int s_item, s_ph, s_b, s_t, s_q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = kSolveThreads / 32;
    const int nblk = cdiv(n, NB), ntile = cdiv(n, TR);
    const int total = off[2 * nblk];
    int bs_key = -1;                                 // which block Bs holds: (ph * 2 + kind) * nblk + b
    for (;;) {
        if (tid == 0) {
            const int item = atomicAdd(&sy->next, 1);
            int ph = 0, b = 0, t = -1, q = 0;
            if (item < total) {
                int lo = 0, hi = 2 * nblk - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= item) lo = mid; else hi = mid - 1;
                }
                const int k = item - off[lo];
                ph = lo < nblk ? 0 : 1;
                b = ph == 0 ? lo : nblk - 1 - (lo - nblk);
                const int parts = cdiv(min(NB, n - b * NB), TR);
                if (k < parts) q = k;
                else t = ph == 0 ? (b + 1) * TPB + (k - parts) : b * TPB - 1 - (k - parts);
            }
            s_item = item;
            s_ph = ph;
            s_b = b;
            s_t = t;
            s_q = q;
        }
        __syncthreads();
        if (s_item >= total) break;
        const int ph = s_ph, b = s_b, t = s_t, q = s_q;
        const int r0 = b * NB, nb = min(NB, n - r0), parts = cdiv(nb, TR);
        const bool part = t < 0;
        // 1. the coefficient rows (independent of everything in flight)
        const int ra = part ? r0 + q * TR : t * TR;      // first output row
        const int nr = min(TR, (part ? r0 + nb : n) - ra);
        if (part) {
            const T* D = DT + (static_cast<size_t>(b) * 2 + ph) * NB * NB;   // D[p][i] = inv[i][p]
            for (int p = warp; p < nb; p += nwarp)
                if (lane < nr) Ls[lane * (NB + 1) + p] = D[static_cast<size_t>(p) * NB + q * TR + lane];
        } else if (chol && ph == 1) {
            // U[ra + i][r0 + p] = L[r0 + p][ra + i]: lanes along the L row
            for (int p = warp; p < nb; p += nwarp)
                if (lane < nr) Ls[lane * (NB + 1) + p] = LU[idx(r0 + p, ra + lane, lda)];
        } else {
            for (int i = warp; i < nr; i += nwarp)
                for (int p = lane; p < nb; p += 32) Ls[i * (NB + 1) + p] = LU[idx(ra + i, r0 + p, lda)];
        }
        // 2. dependencies, all on earlier items
        if (tid == 0) {
            // test hook: the first item also waits on a counter nothing increments
            if (inject && s_item == 0) solve_wait(&sy->pad[0], 1, sy, wait_ns);
            if (part) {
                const int kb = ph == 0 ? b : nblk - 1 - b;
                for (int u = b * TPB; u < min(ntile, (b + 1) * TPB); ++u)
                    solve_wait(ph == 0 ? fdone + u : bdone + u, kb, sy, wait_ns);
                if (ph == 1) solve_wait(xpf + b, parts, sy, wait_ns);
            } else {
                solve_wait(ph == 0 ? xpf + b : xpb + b, parts, sy, wait_ns);
                if (ph == 1) {
                    const int tb = t / TPB;
                    solve_wait(xpf + tb, cdiv(min(NB, n - tb * NB), TR), sy, wait_ns);
                }
                solve_wait(ph == 0 ? fdone + t : bdone + t, ph == 0 ? b : nblk - 1 - b, sy, wait_ns);
            }
            __threadfence();
        }
        __syncthreads();
        // 3. the right operand: the block's right-hand side (part) or its solution (tile);
        //    written by other CTAs, so read past L1
        const int key = (ph * 2 + (part ? 0 : 1)) * nblk + b;
        if (bs_key != key) {
            const T* src = part ? (ph == 0 ? Y : X) : (ph == 0 ? X : Y);
            for (int e = tid; e < nb * NCW; e += kSolveThreads) Bs[e] = __ldcg(src + static_cast<size_t>(r0) * NCW + e);
            bs_key = key;
        }
        __syncthreads();
        // 4. 32 rows x NCW: out = Ls Bs
        const int i = tid >> 3, cg = tid & 7;
        T acc[MU];
#pragma unroll
        for (int k = 0; k < MU; ++k) acc[k] = T(0);
        if (i < nr) {
#pragma unroll 4
            for (int p = 0; p < nb; ++p) {
                const T l = Ls[i * (NB + 1) + p];
#pragma unroll
                for (int k = 0; k < MU; ++k) acc[k] = fma(l, Bs[p * NCW + cg + 8 * k], acc[k]);
            }
            if (part) {
                T* row = (ph == 0 ? X : Y) + static_cast<size_t>(ra + i) * NCW;
#pragma unroll
                for (int k = 0; k < MU; ++k) row[cg + 8 * k] = acc[k];
            } else {
                T* row = (ph == 0 ? Y : X) + static_cast<size_t>(ra + i) * NCW;
#pragma unroll
                for (int k = 0; k < MU; ++k) row[cg + 8 * k] = __ldcg(row + cg + 8 * k) - acc[k];
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (part) atomicAdd(ph == 0 ? xpf + b : xpb + b, 1);
            else atomicAdd(ph == 0 ? fdone + t : bdone + t, 1);
        }
    }
}

template <typename T, int NCW>
static size_t solve_smem() {
    constexpr int NB = SolveNB<T>::value;
    return (static_cast<size_t>(kSolveTile) * (NB + 1) + static_cast<size_t>(NB) * NCW) * sizeof(T);
}

// CTAs of the item kernel: as many as fit on the device, up to 4 per SM
// (none need to be resident together).
template <typename T, int NCW>
static int solve_grid() {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = solve_smem<T, NCW>();
    if (smem_attr(solve_items_kernel<T, NCW>, smem) != 0) return -1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_items_kernel<T, NCW>, kSolveThreads, smem);
    cudaGetLastError();
    if (per < 1 || sms < 1) return -1;
    return sms * (per < 4 ? per : 4);
}

template <typename T, int NCW>
static int solve_launch(int n, const SolvePlan<T>& p, T* Y, T* X, int* fdone, int* bdone, int* xpf, int* xpb,
                        SolveSync* sy, cudaStream_t s) {
    const int G = solve_grid<T, NCW>();
    if (G <= 0) return LU_EUNSUPPORTED;
    const WaitCfg wc = wait_cfg(LU_WAIT_SITE_SOLVE);
    solve_items_kernel<T, NCW><<<G, kSolveThreads, solve_smem<T, NCW>(), s>>>(
        n, p.LU, p.lda, p.DT, p.off, Y, X, fdone, bdone, xpf, xpb, sy, p.chol, wc.wait_ns, wc.inject);
    count_launches(1);
    return 0;
}

// gather with zero padding: Y[i][c] = B[perm[i]][c0 + c] for c < nc, 0 for nc <= c < w
template <typename T>
__global__ void gather_rows_pad(int n, int nc, int w, const int* __restrict__ perm, const T* __restrict__ B, int ldb,
                                T* __restrict__ Y) {
    const long long tot = static_cast<long long>(n) * w;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / w), c = static_cast<int>(e % w);
        Y[e] = c < nc ? B[idx(perm[i], c, ldb)] : T(0);
    }
}

template <typename T>
__global__ void copy_out_pad(int n, int nc, int w, const T* __restrict__ Y, T* __restrict__ B, int ldb) {
    const long long tot = static_cast<long long>(n) * nc;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / nc), c = static_cast<int>(e % nc);
        B[idx(i, c, ldb)] = Y[static_cast<size_t>(i) * w + c];
    }
}

__global__ void perm_identity(int n, int* __restrict__ perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

// piv == nullptr: LU holds a Cholesky factor L (lower triangle), solved as
// L (L^T X) = B with no permutation.
template <typename T>
int solve_plan_make(int n, const T* LU, int lda, const int* piv, SolvePlan<T>* p, cudaStream_t s) {
    constexpr int NB = SolveNB<T>::value;
    *p = SolvePlan<T>{};
    p->n = n;
    p->LU = LU;
    p->lda = lda;
    p->chol = piv == nullptr ? 1 : 0;
    if (n == 0) return 0;
    const int nblk = cdiv(n, NB);
    if (cudaMallocAsync(reinterpret_cast<void**>(&p->perm), sizeof(int) * static_cast<size_t>(n), s) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&p->DT), sizeof(T) * static_cast<size_t>(nblk) * 2 * NB * NB, s) !=
            cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&p->off), sizeof(int) * (2 * static_cast<size_t>(nblk) + 1), s) !=
            cudaSuccess) {
        cudaGetLastError();
        solve_plan_free(p, s);
        return LU_ENOMEM;
    }
    if (p->chol) {
        ProfScope ps(LU_PROF_SOLVE, s);
        perm_identity<<<cdiv(n, 256) < 1024 ? cdiv(n, 256) : 1024, 256, 0, s>>>(n, p->perm);
        count_launches(1);
    } else if (n <= kPermSmemMax) {
        const size_t smem = static_cast<size_t>(n) * sizeof(int);
        if (int rc_ = smem_attr(perm_from_piv_smem, smem)) return rc_;
        ProfScope ps(LU_PROF_SOLVE, s);
        perm_from_piv_smem<<<1, 256, smem, s>>>(n, piv, p->perm);
        count_launches(1);
    } else {
        ProfScope ps(LU_PROF_SOLVE, s);
        perm_from_piv_global<<<1, 256, 0, s>>>(n, piv, p->perm);
        count_launches(1);
    }
    LU_LAUNCHED();
    {
        const size_t ismem = 2 * static_cast<size_t>(NB) * (NB + 1) * sizeof(T);
        if (int rc_ = smem_attr(invert_diag_kernel<T>, ismem)) return rc_;
        ProfScope ps(LU_PROF_SOLVE, s);
        invert_diag_kernel<T><<<dim3(nblk, 2), 128, ismem, s>>>(n, LU, lda, p->DT, p->chol);
        count_launches(1);
    }
    LU_LAUNCHED();
    {
        const int nbv = NB;
        LU_TRY(cudaMemcpyAsync(p->off, &nbv, sizeof(int), cudaMemcpyHostToDevice, s));
        ProfScope ps(LU_PROF_SOLVE, s);
        solve_offsets_kernel<<<1, 32, 0, s>>>(n, p->off);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template <typename T>
void solve_plan_free(SolvePlan<T>* p, cudaStream_t s) {
    if (p->perm) cudaFreeAsync(p->perm, s);
    if (p->DT) cudaFreeAsync(p->DT, s);
    if (p->off) cudaFreeAsync(p->off, s);
    p->perm = nullptr;
    p->DT = nullptr;
    p->off = nullptr;
}

template <typename T>
int solve_plan_apply(const SolvePlan<T>& p, int nrhs, T* B, int ldb, cudaStream_t s) {
    constexpr int NB = SolveNB<T>::value;
    const int n = p.n;
    if (n == 0 || nrhs == 0) return 0;
    const int nblk = cdiv(n, NB), ntile = cdiv(n, kSolveTile);
    const size_t vs = static_cast<size_t>(n) * kSolveRhs;
    const size_t flags = sizeof(SolveSync) + sizeof(int) * (2 * static_cast<size_t>(ntile) + 2 * nblk);
    const size_t fbytes = (flags + 255) / 256 * 256;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, fbytes + sizeof(T) * 2 * vs, s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    SolveSync* sy = static_cast<SolveSync*>(ws);
    int* fdone = reinterpret_cast<int*>(sy + 1);
    int* bdone = fdone + ntile;
    int* xpf = bdone + ntile;
    int* xpb = xpf + nblk;
    T* Y = reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + fbytes);
    T* X = Y + vs;
    int rc = 0;
    int timeout = 0;
    for (int c0 = 0; c0 < nrhs && !rc; c0 += kSolveRhs) {
        const int nc = (nrhs - c0) < kSolveRhs ? (nrhs - c0) : kSolveRhs;
        const int w = nc <= 8 ? 8 : nc <= 16 ? 16 : nc <= 32 ? 32 : 64;
        const long long tot = static_cast<long long>(n) * w;
        const int gblocks = static_cast<int>(tot / 256 + 1 < 4096 ? tot / 256 + 1 : 4096);
        if (cudaMemsetAsync(ws, 0, flags, s) != cudaSuccess) {
            rc = LU_ELAUNCH;
            break;
        }
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            gather_rows_pad<T><<<gblocks, 256, 0, s>>>(n, nc, w, p.perm, B + c0, ldb, Y);
            count_launches(1);
        }
        {
            ProfScope ps(LU_PROF_SOLVE, s, 2.0 * static_cast<double>(n) * n * nc);
            rc = w == 8    ? solve_launch<T, 8>(n, p, Y, X, fdone, bdone, xpf, xpb, sy, s)
                 : w == 16 ? solve_launch<T, 16>(n, p, Y, X, fdone, bdone, xpf, xpb, sy, s)
                 : w == 32 ? solve_launch<T, 32>(n, p, Y, X, fdone, bdone, xpf, xpb, sy, s)
                           : solve_launch<T, 64>(n, p, Y, X, fdone, bdone, xpf, xpb, sy, s);
        }
        if (rc) break;
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            copy_out_pad<T><<<gblocks, 256, 0, s>>>(n, nc, w, Y, B + c0, ldb);
            count_launches(1);
        }
        if (cudaPeekAtLastError() != cudaSuccess) {
            cudaGetLastError();
            rc = LU_ELAUNCH;
            break;
        }
        int to = 0;
        if (cudaMemcpyAsync(&to, &sy->timeout, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = LU_ELAUNCH;
            break;
        }
        timeout |= to;
    }
    if (!rc && timeout) rc = LU_ETIMEOUT;
    cudaFreeAsync(ws, s);
    return rc;
}

template <typename T>
int getrs_alloc(int n, int nrhs, const T* LU, int lda, const int* piv, T* B, int ldb, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return 0;
    SolvePlan<T> p;
    int rc = solve_plan_make<T>(n, LU, lda, piv, &p, s);
    if (!rc) rc = solve_plan_apply<T>(p, nrhs, B, ldb, s);
    solve_plan_free<T>(&p, s);
    return rc;
}

template int solve_plan_make<float>(int, const float*, int, const int*, SolvePlan<float>*, cudaStream_t);
template int solve_plan_apply<float>(const SolvePlan<float>&, int, float*, int, cudaStream_t);
template void solve_plan_free<float>(SolvePlan<float>*, cudaStream_t);

int getrs_f64(int n, int nrhs, const double* LU, int lda, const int* piv, double* B, int ldb, cudaStream_t s) {
    return getrs_alloc<double>(n, nrhs, LU, lda, piv, B, ldb, s);
}

int getrs_f32(int n, int nrhs, const float* LU, int lda, const int* piv, float* B, int ldb, cudaStream_t s) {
    return getrs_alloc<float>(n, nrhs, LU, lda, piv, B, ldb, s);
}

}  // namespace lu

using namespace lu;

// Cholesky solve: the same work-list substitution with L and L^T.
template <typename T>
static int chol_solve_t(int n, int nrhs, const T* L, int lda, T* B, int ldb, cudaStream_t s) {
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > 384) return -2;
    if (n > 0 && L == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && nrhs > 0 && B == nullptr) return -5;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -6;
    return getrs_alloc<T>(n, nrhs, L, lda, nullptr, B, ldb, s);
}

extern "C" int chol_solve(int n, int nrhs, const double* L, int lda, double* B, int ldb, cudaStream_t stream) {
    return chol_solve_t<double>(n, nrhs, L, lda, B, ldb, stream);
}

extern "C" int chol_solve_f32(int n, int nrhs, const float* L, int lda, float* B, int ldb, cudaStream_t stream) {
    return chol_solve_t<float>(n, nrhs, L, lda, B, ldb, stream);
}

