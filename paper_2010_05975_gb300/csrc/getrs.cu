// Solve A X = B with the factors P A = L U (getrs): X = U^{-1} L^{-1} P B.
// The linear solve is what the paper's factorization serves ("linear
// solvers", Section 1); the paper does not spell it out.  A Cholesky factor
// L goes through the same machinery with U = L^T and no permutation.
//
// A solve plan holds what depends on the factors only: the row permutation
// composed from the swap sequence piv, and the inverses of the NB x NB
// diagonal blocks of L (unit lower) and U (upper), and the coupling blocks
// inv(L_bb) L_{b,b-1} and inv(U_bb) U_{b,b+1}, all stored row-major.  The
// refinement keeps one plan per factorization; the one-shot entry points
// build and drop one per call.
//
// Applying a plan: B is gathered through the permutation into Y (row stride
// nc, padded to a width of 8, 16, 32 or 64), then one kernel runs the
// blocked forward and backward substitutions as a list of work items taken
// in order from an atomic counter.  Per block b the list holds
//   the chain item  forward:  X_b = inv(L_bb) Y_b - M_b X_{b-1} with the
//                   plan's coupling block M_b = inv(L_bb) L_{b,b-1};
//                   backward: Y_b = inv(U_bb) X_b - M'_b Y_{b+1}, M'_b =
//                   inv(U_bb) U_{b,b+1} (b from the last block up).  The
//                   first product needs only the block's earlier updates, so
//                   it runs before the previous chain item is done: one
//                   product per step on the critical path.  It sits in the list
//                   right after the block items of two steps back, a step
//                   ahead of the bulk (solve_offsets_kernel);
//   block items     forward:  for every block t two or more blocks below:
//                   Y_t -= L_tb X_b;  backward: two or more blocks above:
//                   X_t -= U_tb Y_b.
// An item first stages its coefficient blocks (16-byte asynchronous copies
// where the rows are aligned), then waits (bounded, through per-block
// counters) on items earlier in the list, which CTAs already running have
// taken, so the kernel progresses whatever number of its CTAs is resident.
// Each block takes its updates one step at a time, in step order, each as
// y - sum_p l_p x_p with the sum in p order, and every product has a fixed
// order, so results do not depend on timing.  Right-hand sides go through in
// passes of up to 64.
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

// One CTA per (block, factor): Dinv[blk][kind] = inv(diag block), row-major.  Thread c
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
    // row-major: out[i][p] = inv[i][p] (rows arrive in the solve by 16-byte copies)
    T* out = Dinv + (static_cast<size_t>(blk) * 2 + kind) * NB * NB;
    if (chol && kind == 1) {
        // out[i][p] = inv(L^T)[i][p] = inv(L)[p][i]
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = Xs[(e % NB) * (NB + 1) + (e / NB)];
    } else {
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = Xs[(e / NB) * (NB + 1) + (e % NB)];
    }
}

// One CTA per (block, factor): M[blk][kind] = inv(diag block) times the
// off-diagonal block next to it on the substitution's path (kind 0: L_{b,b-1},
// kind 1: U_{b,b+1}; a Cholesky factor's U_{b,b+1} is L_{b+1,b}^T), row-major,
// zero where it has no neighbour.  Fixed summation order.
template <typename T>
__global__ void __launch_bounds__(256) couple_kernel(int n, const T* __restrict__ LU, int lda,
                                                     const T* __restrict__ Dinv, T* __restrict__ M, int chol) {
    constexpr int NB = SolveNB<T>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ds = reinterpret_cast<T*>(smem_raw);              // NB x (NB+1)
    T* Gs = Ds + NB * (NB + 1);                          // NB x (NB+1): the off-diagonal block
    const int blk = blockIdx.x, kind = blockIdx.y;
    const int nblk = cdiv(n, NB);
    const int r0 = blk * NB, nb = min(NB, n - r0);
    const int nbk = kind == 0 ? blk - 1 : blk + 1;
    T* out = M + (static_cast<size_t>(blk) * 2 + kind) * NB * NB;
    if (nbk < 0 || nbk >= nblk) {
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = T(0);
        return;
    }
    const int c0 = nbk * NB, nc = min(NB, n - c0);
    const T* D = Dinv + (static_cast<size_t>(blk) * 2 + kind) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        Ds[i * (NB + 1) + j] = D[e];
        T g = T(0);
        if (i < nb && j < nc) g = (chol && kind == 1) ? LU[idx(c0 + j, r0 + i, lda)] : LU[idx(r0 + i, c0 + j, lda)];
        Gs[i * (NB + 1) + j] = g;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        T acc = T(0);
        for (int q = 0; q < nb; ++q) acc = fma(Ds[i * (NB + 1) + q], Gs[q * (NB + 1) + j], acc);
        out[e] = acc;
    }
}

constexpr int kSolveRhs = 64;            // right-hand sides per pass
constexpr int kSolveThreads = 512;

// Item list bookkeeping (device memory, zeroed before each pass).
struct SolveSync {
    int next;          // next item to take
    int timeout;
    int pad[2];
};

// Item groups: off[g] = first item of group g, g < 2 nblk, off[2 nblk] =
// total; built once per plan (the block size arrives in off[0]).  Forward
// group 0 = {C(0)}, group 1 = {C(1)}, group g >= 2 = {T(g-2, t) for blocks
// t = g .. nblk-1, then C(g)}: the chain item of block g follows the block
// items of step g-2, so it is taken (and stages its coefficients) a step
// ahead of the bulk of step g-1.  Backward groups mirror it from the last
// block: group g holds C'(nblk-1-g) after T'(nblk+1-g, t) for t = nblk-1-g
// down to 0.
__global__ void solve_offsets_kernel(int n, int* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int NB = off[0];
    const int nblk = cdiv(n, NB);
    int acc = 0;
    for (int g = 0; g < nblk; ++g) {                    // forward
        off[g] = acc;
        acc += g < 2 ? 1 : nblk - g + 1;
    }
    for (int g = 0; g < nblk; ++g) {                    // backward: block b = nblk - 1 - g
        off[nblk + g] = acc;
        acc += g < 2 ? 1 : nblk - g + 1;
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

// Stage rows x cols of a row-major block (leading dimension ld) into shared
// memory with row pitch cp, zero outside [0, vrows) x [0, vcols): 16-byte
// asynchronous copies when vec (every staged row 16-byte aligned; cp a
// multiple of 16 bytes), else plain loads.  The caller waits and syncs.
template <typename T>
__device__ __forceinline__ void solve_stage(T* dst, int cp, const T* src, size_t ld, int rows, int cols, int vrows,
                                            int vcols, bool vec) {
    constexpr int V = 16 / static_cast<int>(sizeof(T));
    if (vec) {
        const int cq = cols / V;
        for (int e = threadIdx.x; e < rows * cq; e += kSolveThreads) {
            const int r = e / cq, c = V * (e - r * cq);
            const int bytes = (r < vrows) ? static_cast<int>(sizeof(T)) * max(0, min(V, vcols - c)) : 0;
            cp_async16(dst + static_cast<size_t>(r) * cp + c, bytes ? src + r * ld + c : src, bytes);
        }
    } else {
        for (int e = threadIdx.x; e < rows * cols; e += kSolveThreads) {
            const int r = e / cols, c = e - r * cols;
            dst[static_cast<size_t>(r) * cp + c] = (r < vrows && c < vcols) ? src[r * ld + c] : T(0);
        }
    }
}

// The transposed block (a Cholesky factor's U = L^T): dst[i][p] = src[p][i].
template <typename T>
__device__ __forceinline__ void solve_stage_t(T* dst, int cp, const T* src, size_t ld, int rows, int cols) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = warp; p < cols; p += kSolveThreads / 32)
        for (int i = lane; i < rows; i += 32) dst[static_cast<size_t>(i) * cp + p] = src[p * ld + i];
}

// out[i][c] (op) = sum_{p < np} C[i][p] * Bm[p][c] for rows i < nr, p in
// order.  A thread sums a 4 x 4 tile (rows rg, rg + NB/4, rg + NB/2,
// rg + 3 NB/4, columns 4 cg..): per four p it reads four 16-byte pieces of C
// rows and four of Bm rows for 64 multiply-adds, the ratio that keeps the
// shared-memory reads (their bytes into registers, not the multiply-adds,
// bound these small products) low; a warp's eight row groups are
// consecutive rows, whose 16-byte pieces fall in distinct bank groups (row
// pitch an odd number of 16-byte chunks).  C row pitch cp and Bm row pitch
// NCW give 16-byte aligned rows.  sub: out = base - sum; else out = sum.
template <typename T>
__device__ __forceinline__ void solve_ld4(const T* p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2*>(p);
        const double2 y = *reinterpret_cast<const double2*>(p + 2);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = y.x;
        v[3] = y.y;
    }
}

template <typename T, int NCW>
__device__ __forceinline__ void solve_rows(const T* C, int cp, const T* Bm, int nr, int np, const T* base, int bstride,
                                           T* out, int ostride, bool sub) {
    constexpr int NB = SolveNB<T>::value;
    constexpr int RB = 4;                              // rows per thread
    constexpr int CG = NCW / 4;                        // column groups of four
    constexpr int NT = (NB / RB) * CG;                 // threads in use
    static_assert(NT <= kSolveThreads, "one thread per (row group, column group)");
    constexpr int RS = NB / RB;                        // row stride: rows rg, rg + RS, ...
    if (threadIdx.x >= NT) return;
    const int cg = threadIdx.x % CG, rg = threadIdx.x / CG;
    const int c = 4 * cg;
    if (rg >= nr) return;
    T acc[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[r][k] = T(0);
    const T* Cr = C + static_cast<size_t>(rg) * cp;
    const int np4 = np & ~3;
    for (int p = 0; p < np4; p += 4) {
        T cv[RB][4];
#pragma unroll
        for (int r = 0; r < RB; ++r) solve_ld4(Cr + r * RS * cp + p, cv[r]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T bv[4];
            solve_ld4(Bm + (p + q) * NCW + c, bv);
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[r][k] = fma(cv[r][q], bv[k], acc[r][k]);
        }
    }
    for (int p = np4; p < np; ++p) {
        T bv[4];
        solve_ld4(Bm + p * NCW + c, bv);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[r][k] = fma(Cr[r * RS * cp + p], bv[k], acc[r][k]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (rg + r * RS >= nr) break;
        const size_t i = static_cast<size_t>(rg + r * RS);
#pragma unroll
        for (int k = 0; k < 4; ++k) out[i * ostride + c + k] = sub ? base[i * bstride + c + k] - acc[r][k] : acc[r][k];
    }
}

// Coefficient row pitch: a whole number of 16-byte chunks plus one.
template <typename T>
__host__ __device__ constexpr int solve_cp() {
    return SolveNB<T>::value + 16 / static_cast<int>(sizeof(T));
}

// Forward (L: Y -> X) then backward (U: X -> Y) substitution; right-hand
// sides row-major with stride NCW (columns >= nc are zero and stay zero).
// With chol set, U is L^T: the backward coefficients read L transposed.
// xpf[b] / xpb[b]: the chain item of block b is done; fdone[t] / bdone[t]:
// block items applied to block t.  vec: LU's rows are 16-byte aligned.
template <typename T, int NCW>
__global__ void __launch_bounds__(kSolveThreads) solve_items_kernel(int n, const T* __restrict__ LU, int lda,
                                                                    const T* __restrict__ DM,
                                                                    const T* __restrict__ MM,
                                                                    const int* __restrict__ off, T* Y, T* X,
                                                                    int* fdone, int* bdone, int* xpf, int* xpb,
                                                                    SolveSync* sy, int chol, int vec,
                                                                    unsigned long long wait_ns, int inject) {
    constexpr int NB = SolveNB<T>::value;
    constexpr int CP = solve_cp<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Cs = reinterpret_cast<T*>(smem_raw);          // NB x CP: off-diagonal coefficients
    T* Ds = Cs + NB * CP;                            // NB x CP: inverse of the diagonal block (chain)
    T* Bs = Ds + NB * CP;                            // NB x NCW: the neighbour's solution
    T* Ws = Bs + NB * NCW;                           // NB x NCW: the block's current values
    __shared__ int s_item, s_ph, s_b, s_t;
    const int tid = threadIdx.x;
    const int nblk = cdiv(n, NB);
    const int total = off[2 * nblk];
    for (;;) {
        if (tid == 0) {
            const int item = atomicAdd(&sy->next, 1);
            int ph = 0, b = 0, t = -1;
            if (item < total) {
                int lo = 0, hi = 2 * nblk - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= item) lo = mid; else hi = mid - 1;
                }
                const int k = item - off[lo];
                const int g = lo < nblk ? lo : lo - nblk;     // group within the phase
                const int nbi = g < 2 ? 0 : nblk - g;          // block items before the chain item
                ph = lo < nblk ? 0 : 1;
                if (k == nbi) {                                // the chain item of block g (forward) / nblk-1-g
                    b = ph == 0 ? g : nblk - 1 - g;
                } else if (ph == 0) {                          // T(g-2, g + k)
                    b = g - 2;
                    t = g + k;
                } else {                                       // T'(nblk+1-g, nblk-1-g-k)
                    b = nblk + 1 - g;
                    t = nblk - 1 - g - k;
                }
            }
            s_item = item;
            s_ph = ph;
            s_b = b;
            s_t = t;
        }
        __syncthreads();
        if (s_item >= total) break;
        const int ph = s_ph, b = s_b, t = s_t;
        const bool chain = t < 0;
        const int r0 = (chain ? b : t) * NB, nr = min(NB, n - r0);          // rows this item writes
        // coefficient columns: the neighbour block (chain) or block b (block item); -1: none
        const int cb = chain ? (ph == 0 ? b - 1 : (b + 1 < nblk ? b + 1 : -1)) : b;
        const int c0 = cb * NB, nc = cb >= 0 ? min(NB, n - c0) : 0;
        // 1. coefficients (independent of everything in flight)
        if (chain) {
            solve_stage(Ds, CP, DM + (static_cast<size_t>(b) * 2 + ph) * NB * NB, NB, NB, NB, nr, nr, true);
            if (cb >= 0) solve_stage(Cs, CP, MM + (static_cast<size_t>(b) * 2 + ph) * NB * NB, NB, NB, NB, nr, nc, true);
        } else if (chol && ph == 1) {
            solve_stage_t(Cs, CP, LU + idx(c0, r0, lda), lda, nr, nc);              // U[r0+i][c0+p] = L[c0+p][r0+i]
        } else {
            solve_stage(Cs, CP, LU + idx(r0, c0, lda), lda, NB, NB, nr, nc, vec != 0);
        }
        // 2. dependencies on earlier items: the rows' own earlier updates (and,
        //    backward, their forward values) first
        if (tid == 0) {
            // test hook: the first item also waits on a counter nothing increments
            if (inject && s_item == 0) solve_wait(&sy->pad[0], 1, sy, wait_ns);
            if (chain) {
                if (ph == 0) {
                    solve_wait(fdone + b, b - 1, sy, wait_ns);
                } else {
                    solve_wait(xpf + b, 1, sy, wait_ns);                     // forward X_b
                    solve_wait(bdone + b, nblk - b - 2, sy, wait_ns);
                }
            } else if (ph == 0) {
                solve_wait(xpf + b, 1, sy, wait_ns);
                solve_wait(fdone + t, b, sy, wait_ns);
            } else {
                solve_wait(xpb + b, 1, sy, wait_ns);
                solve_wait(xpf + t, 1, sy, wait_ns);                         // forward X_t
                solve_wait(bdone + t, nblk - 1 - b, sy, wait_ns);
            }
            __threadfence();
        }
        __syncthreads();
        // 3. operands written by other CTAs: 16-byte asynchronous copies, which
        //    read through L2 only (the waits above ordered them after the writers)
        solve_stage(Ws, NCW, (ph == 0 ? Y : X) + static_cast<size_t>(r0) * NCW, NCW, nr, NCW, nr, NCW, true);
        if (!chain) solve_stage(Bs, NCW, (ph == 0 ? X : Y) + static_cast<size_t>(c0) * NCW, NCW, nc, NCW, nc, NCW, true);
        cp_async_wait_all();
        __syncthreads();
        // 4. products
        T* dst = (ph == 0 ? (chain ? X : Y) : (chain ? Y : X)) + static_cast<size_t>(r0) * NCW;
        if (chain) {
            solve_rows<T, NCW>(Ds, CP, Ws, nr, nr, nullptr, 0, dst, NCW, false);   // inv(diag) times the rows
            if (cb >= 0) {
                // the neighbour's solution (the previous chain item), then the coupling
                if (tid == 0) {
                    solve_wait(ph == 0 ? xpf + cb : xpb + cb, 1, sy, wait_ns);
                    __threadfence();
                }
                __syncthreads();
                solve_stage(Bs, NCW, (ph == 0 ? X : Y) + static_cast<size_t>(c0) * NCW, NCW, nc, NCW, nc, NCW, true);
                cp_async_wait_all();
                __syncthreads();
                // each thread reads back the entries it wrote above (same thread mapping)
                solve_rows<T, NCW>(Cs, CP, Bs, nr, nc, dst, NCW, dst, NCW, true);
            }
        } else {
            solve_rows<T, NCW>(Cs, CP, Bs, nr, nc, Ws, NCW, dst, NCW, true);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (chain) atomicAdd(ph == 0 ? xpf + b : xpb + b, 1);
            else atomicAdd(ph == 0 ? fdone + t : bdone + t, 1);
        }
    }
}

constexpr int kPartsTile = 32;           // rows per part / tile of the binary64 list
constexpr int kPartsThreads = 256;

// The binary64 list: items before forward step b / backward step b,
// off[0..2*nblk], built once per plan (the block size arrives in off[0]).
// Step b: the 32-row parts of the diagonal solve, then every tile below
// (forward) or above (backward).
__global__ void solve_parts_offsets_kernel(int n, int* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    constexpr int TR = kPartsTile;
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

// The binary64 substitution (the DFMA pipe, about 2 per clock per SM, makes a
// one-CTA chain step slow, so a step's diagonal solve is split into 32-row
// parts on several CTAs): forward (L: Y -> X) then backward (U: X -> Y);
// right-hand sides row-major with stride NCW (columns >= nc are zero and
// stay zero).  With chol set, U is L^T: the backward tiles read L
// transposed.
template <typename T, int NCW>
__global__ void __launch_bounds__(kPartsThreads) solve_parts_kernel(int n, const T* __restrict__ LU, int lda,
                                                                    const T* __restrict__ DT,
                                                                    const int* __restrict__ off, T* Y, T* X,
                                                                    int* fdone, int* bdone, int* xpf, int* xpb,
                                                                    SolveSync* sy, int chol,
                                                                    unsigned long long wait_ns, int inject) {
    constexpr int NB = SolveNB<T>::value;
    constexpr int TR = kPartsTile;
    constexpr int TPB = NB / TR;                     // tiles (and solve parts) per block
    constexpr int MU = NCW / 8;                      // columns per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ls = reinterpret_cast<T*>(smem_raw);          // TR x (NB+1): the item's coefficient rows
    T* Bs = Ls + TR * (NB + 1);                      // NB x NCW: the right operand
    __shared__ int s_item, s_ph, s_b, s_t, s_q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = kPartsThreads / 32;
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
            const T* D = DT + (static_cast<size_t>(b) * 2 + ph) * NB * NB;   // D[i][p] = inv[i][p]
            for (int i = warp; i < nr; i += nwarp)
                for (int p = lane; p < nb; p += 32) Ls[i * (NB + 1) + p] = D[static_cast<size_t>(q * TR + i) * NB + p];
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
            for (int e = tid; e < nb * NCW; e += kPartsThreads) Bs[e] = __ldcg(src + static_cast<size_t>(r0) * NCW + e);
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
    if constexpr (sizeof(T) == 8)
        return (static_cast<size_t>(kPartsTile) * (NB + 1) + static_cast<size_t>(NB) * NCW) * sizeof(T);
    return (2 * static_cast<size_t>(NB) * solve_cp<T>() + 2 * static_cast<size_t>(NB) * NCW) * sizeof(T);
}

// CTAs of the item kernel: as many as fit on the device, up to 2 per SM
// (none need to be resident together).
template <typename T, int NCW>
static int solve_grid() {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = solve_smem<T, NCW>();
    if constexpr (sizeof(T) == 8) {
        if (smem_attr(solve_parts_kernel<T, NCW>, smem) != 0) return -1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_parts_kernel<T, NCW>, kPartsThreads, smem);
        cudaGetLastError();
        if (per < 1 || sms < 1) return -1;
        return sms * (per < 4 ? per : 4);
    }
    if (smem_attr(solve_items_kernel<T, NCW>, smem) != 0) return -1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_items_kernel<T, NCW>, kSolveThreads, smem);
    cudaGetLastError();
    if (per < 1 || sms < 1) return -1;
    return sms * (per < 2 ? per : 2);
}

template <typename T, int NCW>
static int solve_launch(int n, const SolvePlan<T>& p, T* Y, T* X, int* fdone, int* bdone, int* xpf, int* xpb,
                        SolveSync* sy, cudaStream_t s) {
    const int G = solve_grid<T, NCW>();
    if (G <= 0) return LU_EUNSUPPORTED;
    const WaitCfg wc = wait_cfg(LU_WAIT_SITE_SOLVE);
    if constexpr (sizeof(T) == 8) {
        solve_parts_kernel<T, NCW><<<G, kPartsThreads, solve_smem<T, NCW>(), s>>>(
            n, p.LU, p.lda, p.DT, p.off, Y, X, fdone, bdone, xpf, xpb, sy, p.chol, wc.wait_ns, wc.inject);
    } else {
        constexpr int V = 16 / static_cast<int>(sizeof(T));
        const int vec = (reinterpret_cast<uintptr_t>(p.LU) & 15) == 0 && (p.lda % V) == 0 ? 1 : 0;
        solve_items_kernel<T, NCW><<<G, kSolveThreads, solve_smem<T, NCW>(), s>>>(
            n, p.LU, p.lda, p.DT, p.M, p.off, Y, X, fdone, bdone, xpf, xpb, sy, p.chol, vec, wc.wait_ns, wc.inject);
    }
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
    if (lu_malloc_async(reinterpret_cast<void**>(&p->perm), sizeof(int) * static_cast<size_t>(n), s) != cudaSuccess ||
        lu_malloc_async(reinterpret_cast<void**>(&p->DT), sizeof(T) * static_cast<size_t>(nblk) * 2 * NB * NB, s) !=
            cudaSuccess ||
        (sizeof(T) == 4 &&
         lu_malloc_async(reinterpret_cast<void**>(&p->M), sizeof(T) * static_cast<size_t>(nblk) * 2 * NB * NB, s) !=
             cudaSuccess) ||
        lu_malloc_async(reinterpret_cast<void**>(&p->off), sizeof(int) * (2 * static_cast<size_t>(nblk) + 1), s) !=
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
    if (sizeof(T) == 4) {
        const size_t csmem = 2 * static_cast<size_t>(NB) * (NB + 1) * sizeof(T);
        if (int rc_ = smem_attr(couple_kernel<T>, csmem)) return rc_;
        ProfScope ps(LU_PROF_SOLVE, s);
        couple_kernel<T><<<dim3(nblk, 2), 256, csmem, s>>>(n, LU, lda, p->DT, p->M, p->chol);
        count_launches(1);
    }
    LU_LAUNCHED();
    {
        const int nbv = NB;
        LU_TRY(cudaMemcpyAsync(p->off, &nbv, sizeof(int), cudaMemcpyHostToDevice, s));
        ProfScope ps(LU_PROF_SOLVE, s);
        if (sizeof(T) == 8)
            solve_parts_offsets_kernel<<<1, 32, 0, s>>>(n, p->off);
        else
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
    if (p->M) cudaFreeAsync(p->M, s);
    if (p->off) cudaFreeAsync(p->off, s);
    p->perm = nullptr;
    p->DT = nullptr;
    p->M = nullptr;
    p->off = nullptr;
}

template <typename T>
int solve_plan_apply(const SolvePlan<T>& p, int nrhs, T* B, int ldb, cudaStream_t s) {
    constexpr int NB = SolveNB<T>::value;
    const int n = p.n;
    if (n == 0 || nrhs == 0) return 0;
    const int nblk = cdiv(n, NB), ntile = cdiv(n, kPartsTile);
    const int nflag = sizeof(T) == 8 ? ntile : nblk;           // per-tile (binary64) or per-block counters
    const size_t vs = static_cast<size_t>(n) * kSolveRhs;
    const size_t flags = sizeof(SolveSync) + sizeof(int) * (2 * static_cast<size_t>(nflag) + 2 * nblk);
    const size_t fbytes = (flags + 255) / 256 * 256;
    void* ws = nullptr;
    if (lu_malloc_async(&ws, fbytes + sizeof(T) * 2 * vs, s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    SolveSync* sy = static_cast<SolveSync*>(ws);
    int* fdone = reinterpret_cast<int*>(sy + 1);
    int* bdone = fdone + nflag;
    int* xpf = bdone + nflag;
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

