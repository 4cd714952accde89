// Blocked GEPP candidate selection for a tournament node held by one CTA
// (the local LUP of TournPivot, Section 7.3).  Used by the tree kernel's
// one-CTA nodes and by the batched factorization.
//
// The node's nr rows sit in shared memory W (row stride gepp_ws<T>(w)), in
// ascending order of row position.  Pivots are chosen KB columns at a time:
//   panel phase  the warps that hold rows (one thread per row) keep the
//                row's KB panel values in registers.  Per column: warp
//                argmax by two reductions (largest |a|, then lowest lane),
//                the warp's candidate writes its key and KB values to a
//                slot, one barrier among those warps, every thread folds
//                the slots the same way and reads the winner's values,
//                then divides and updates in registers.  The winner's
//                bookkeeping waits for the end of the panel.
//   triangle     the panel warps update the pivot rows' trailing columns
//                (one thread per column) with the pivot rows' multipliers:
//                binary32 takes the ones each thread read at their steps,
//                binary64 (register pressure) reads them back from W after
//                one more barrier among those warps.
//   rank-KB      every thread takes 16-byte chunks of one unchosen row's
//                trailing columns and applies the KB updates.
// Every element still receives a = fma(-l, u, a) for its pivots in
// ascending order, each multiplier is one IEEE division, and a step whose
// pivot is zero updates nothing, so the result is the column-by-column GEPP
// bit for bit.  Ties in |a| go to the lowest row, that is the smallest row
// position; a NaN counts as +inf, so every step has a pivot row.
#pragma once
#include <climits>
#include <cuda_runtime.h>

namespace lu {

constexpr int kGeppKB = 8;   // columns per panel of the blocked node GEPP

// Row stride in elements: a whole number of KB-column panels plus 16 bytes,
// so rows start 16-byte aligned and their stride is an odd multiple of 16
// bytes (a quarter-warp's 16-byte accesses to 8 consecutive rows hit 8
// distinct bank groups).
template <typename T>
__host__ __device__ constexpr int gepp_ws(int w) {
    return (w + kGeppKB - 1) / kGeppKB * kGeppKB + 16 / static_cast<int>(sizeof(T));
}

// Per-warp candidates of one column step (double-buffered) and the panel's
// zero-pivot mask.
template <typename T>
struct GeppSlots {
    int key[2][32];             // |a| key: binary32 bits, or the high word of binary64
    unsigned key_lo[2][32];     // binary64: low word
    int row[2][32];
    alignas(16) T val[2][32][kGeppKB];
    unsigned zm;
};

// Pivot key of a live row: the bits of |a| (monotone in |a|), NaN clamped
// to +inf; -1 for a row that is not a candidate.
__device__ __forceinline__ void gepp_key(float x, bool live, int& hi, unsigned& lo) {
    hi = live ? min(__float_as_int(x) & 0x7fffffff, 0x7f800000) : -1;
    lo = 0u;
}
__device__ __forceinline__ void gepp_key(double x, bool live, int& hi, unsigned& lo) {
    const long long b = min(__double_as_longlong(x) & 0x7fffffffffffffffLL, 0x7ff0000000000000LL);
    hi = live ? static_cast<int>(b >> 32) : -1;
    lo = live ? static_cast<unsigned>(b) : 0u;
}

// Largest key over the warp; returns the lowest lane holding it.
template <typename T>
__device__ __forceinline__ int gepp_warp_best(int hi, unsigned lo, int lane, int& mhi, unsigned& mlo) {
    mhi = __reduce_max_sync(0xffffffffu, hi);
    bool cand = (hi == mhi);
    mlo = 0u;
    if (sizeof(T) == 8) {
        mlo = __reduce_max_sync(0xffffffffu, cand ? lo : 0u);
        cand = cand && (lo == mlo);
    }
    return __reduce_min_sync(0xffffffffu, cand ? lane : 32);
}

template <typename T>
__device__ __forceinline__ void gepp_ld16(const T* p, T (&v)[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
}
template <typename T>
__device__ __forceinline__ void gepp_st16(T* p, const T (&v)[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// KB consecutive elements (16-byte aligned).
template <typename T>
__device__ __forceinline__ void gepp_vload(const T* p, T (&v)[kGeppKB]) {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int i = 0; i < kGeppKB / V; ++i) {
        T x[V];
        gepp_ld16(p + V * i, x);
#pragma unroll
        for (int e = 0; e < V; ++e) v[V * i + e] = x[e];
    }
}
template <typename T>
__device__ __forceinline__ void gepp_vstore(T* p, const T (&v)[kGeppKB]) {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int i = 0; i < kGeppKB / V; ++i) {
        T x[V];
#pragma unroll
        for (int e = 0; e < V; ++e) x[e] = v[V * i + e];
        gepp_st16(p + V * i, x);
    }
}

// The row's panel columns [c0, c0+kb): a partial panel leaves the trailing
// columns after it untouched.
template <typename T>
__device__ __forceinline__ void gepp_store_panel(T* p, const T (&P)[kGeppKB], int kb) {
    if (kb == kGeppKB) {
        gepp_vstore(p, P);
    } else {
#pragma unroll
        for (int q = 0; q < kGeppKB; ++q)
            if (q < kb) p[q] = P[q];
    }
}

__device__ __forceinline__ void gepp_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Row r of W: its trailing columns from j0 (rounded down to 16 bytes; the
// columns before j0 and from w on are written back unchanged), chunks
// i = s, s+S, ..., each taking the panel's KB updates in pivot order: QB
// pivot rows' chunks are read at a time, then their fused multiply-adds.
// Pivot row q is row rq[q] of Ub (stride us); without FULL, steps q >= kb
// and steps whose pivot was zero (bit q of zm) are skipped.
template <typename T, bool FULL, int QB = kGeppKB>
__device__ __forceinline__ void gepp_rank_row(T* W, int ws, int r, int s, int S, int j0, int w,
                                              const T (&mr)[kGeppKB], const T* Ub, int us,
                                              const int (&rq)[kGeppKB], int kb, unsigned zm) {
    constexpr int KB = kGeppKB;
    constexpr int V = 16 / sizeof(T);
    static_assert(KB % QB == 0, "pivot groups must tile the panel");
    const int cb = j0 & ~(V - 1);
    const int nch = (w - cb + V - 1) / V;
    T* row = W + static_cast<size_t>(r) * ws;
    for (int i = s; i < nch; i += S) {
        const int j = cb + V * i;
        T a[V], a0[V];
        gepp_ld16(row + j, a);
#pragma unroll
        for (int v = 0; v < V; ++v) a0[v] = a[v];
#pragma unroll
        for (int q0 = 0; q0 < KB; q0 += QB) {
            T u[QB][V];
#pragma unroll
            for (int t = 0; t < QB; ++t) {
                const int q = q0 + t;
                if (FULL || (q < kb && !((zm >> q) & 1u))) gepp_ld16(Ub + static_cast<size_t>(rq[q]) * us + j, u[t]);
            }
#pragma unroll
            for (int t = 0; t < QB; ++t) {
                const int q = q0 + t;
                if (FULL || (q < kb && !((zm >> q) & 1u))) {
#pragma unroll
                    for (int v = 0; v < V; ++v) a[v] = fma(-mr[q], u[t][v], a[v]);
                }
            }
        }
        if (j < j0 || j + V > w) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (j + v < j0 || j + v >= w) a[v] = a0[v];
        }
        gepp_st16(row + j, a);
    }
}

// GEPP on the node's rows, columns [0, ns) of the w-column panel.
//   W       nr rows in ascending position order, stride ws = gepp_ws<T>(w),
//           16-byte aligned; on return a chosen row holds its multipliers
//           left of its pivot column and its U row from there on, an
//           unchosen row its multipliers in [0, ns) and its reduced values
//           after.  Padding columns [w, ws) are read and written back
//           unchanged.
//   ids     row positions; ord[r] = -1 on entry, on return the step that
//           chose row r, or -1.
//   winp    winp[c] = position of the step-c pivot row; lrow[c] = its row in W.
//   zero_first  if non-null and < 0 on entry: set to the first step whose
//           pivot is zero.
// Requires nr <= blockDim.x (a multiple of 32) and ns <= min(nr, w).  The
// caller has made W, ids and ord visible to the block (a barrier); the
// function ends with a block barrier.  Named barrier 1 is used.
template <typename T, bool LREG = (sizeof(T) == 4), int QB = kGeppKB>
__device__ void node_gepp_blocked(T* W, int ws, int nr, int w, int ns, const int* ids, int* ord, int* winp,
                                  int* lrow, GeppSlots<T>& sl, int* zero_first) {
    constexpr int KB = kGeppKB;
    static_assert(KB % (16 / sizeof(T)) == 0, "panel must be whole 16-byte vectors");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int nwo = (nr + 31) >> 5;                   // warps that hold rows
    const bool own = tid < nr;
    T* const wr = W + static_cast<size_t>(own ? tid : 0) * ws;
    bool live = own && ord[tid] < 0;
    const int myid = own ? ids[tid] : INT_MAX;
    if (ns <= 0) {
        __syncthreads();
        return;
    }
    for (int c0 = 0; c0 < ns; c0 += KB) {
        const int kb = min(KB, ns - c0);
        const int j0 = c0 + kb;
        // ---------------- panel phase, triangle ----------------
        if (warp < nwo) {
            T P[KB];
            if (own) {
                gepp_vload(wr + c0, P);
            } else {
#pragma unroll
                for (int k = 0; k < KB; ++k) P[k] = T(0);
            }
            int khi;
            unsigned klo;
            gepp_key(P[0], live, khi, klo);
            unsigned zm = 0;
            int chosen = -1;
            int rq[KB];
            // LREG (the binary32 default) keeps the step-q pivot row's
            // multipliers L[q][qq] (qq < q) in registers; otherwise they are
            // read back from W.
            constexpr bool kLreg = LREG;
            T L[kLreg ? KB : 1][KB];
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                rq[k] = 0;
                if (k < kb) {
                    const int c = c0 + k;
                    const int buf = c & 1;
                    int mhi;
                    unsigned mlo;
                    const int wl = gepp_warp_best<T>(khi, klo, lane, mhi, mlo);
                    if (lane == wl) {
                        sl.key[buf][warp] = mhi;
                        sl.key_lo[buf][warp] = mlo;
                        sl.row[buf][warp] = tid;
                        gepp_vstore(&sl.val[buf][warp][0], P);
                    }
                    gepp_bar(1, nwo * 32);
                    const int phi = lane < nwo ? sl.key[buf][lane] : -1;
                    const unsigned plo = lane < nwo ? sl.key_lo[buf][lane] : 0u;
                    const int prow = lane < nwo ? sl.row[buf][lane] : INT_MAX;
                    const int ghi = __reduce_max_sync(0xffffffffu, phi);
                    bool cand = (phi == ghi);
                    if (sizeof(T) == 8) {
                        const unsigned glo = __reduce_max_sync(0xffffffffu, cand ? plo : 0u);
                        cand = cand && (plo == glo);
                    }
                    const int lr = __reduce_min_sync(0xffffffffu, cand ? prow : INT_MAX);
                    T U[KB];
                    gepp_vload(&sl.val[buf][lr >> 5][0], U);
                    rq[k] = lr;
                    if constexpr (kLreg) {
#pragma unroll
                        for (int qq = 0; qq < KB; ++qq)
                            if (qq < k) L[k][qq] = U[qq];
                    }
                    const T pv = U[k];
                    const bool pz = (pv == T(0));
                    if (pz) zm |= 1u << k;
                    const bool win = live && (tid == lr);
                    if (win) chosen = k;
                    const bool upd = live && !win && !pz;
                    const T l = P[k] / (upd ? pv : T(1));
                    if (upd) P[k] = l;
#pragma unroll
                    for (int j = k + 1; j < KB; ++j)
                        if (j < kb && upd) P[j] = fma(-l, U[j], P[j]);
                    live = live && !win;
                    gepp_key(P[(k + 1) < KB ? k + 1 : KB - 1], live && k + 1 < kb, khi, klo);
                }
            }
            // the panel's pivot rows: bookkeeping; every live row: its multipliers
            if (chosen >= 0) {
                ord[tid] = c0 + chosen;
                winp[c0 + chosen] = myid;
                lrow[c0 + chosen] = tid;
            }
            if (chosen >= 0 || live) gepp_store_panel(wr + c0, P, kb);
            if (tid == 0) {
                sl.zm = zm;
                if (zero_first != nullptr && zm != 0 && *zero_first < 0) *zero_first = c0 + __ffs(zm) - 1;
            }
            // triangle: the pivot rows' trailing columns, in pivot order
            if constexpr (!kLreg) gepp_bar(1, nwo * 32);  // the pivot rows' multipliers are in W
            if (kb > 1) {
                for (int j = j0 + tid; j < w; j += nwo * 32) {
                    T u[KB];
#pragma unroll
                    for (int q = 0; q < KB; ++q) u[q] = (q < kb) ? W[static_cast<size_t>(rq[q]) * ws + j] : T(0);
#pragma unroll
                    for (int q = 1; q < KB; ++q) {
                        if (q < kb) {
#pragma unroll
                            for (int qq = 0; qq < KB; ++qq) {
                                if (qq < q && !((zm >> qq) & 1u)) {
                                    T lq;
                                    if constexpr (kLreg)
                                        lq = L[q][qq];
                                    else
                                        lq = W[static_cast<size_t>(rq[q]) * ws + c0 + qq];
                                    u[q] = fma(-lq, u[qq], u[q]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 1; q < KB; ++q)
                        if (q < kb) W[static_cast<size_t>(rq[q]) * ws + j] = u[q];
                }
            }
        }
        __syncthreads();
        if (j0 >= w) continue;
        // ---------------- rank-KB update of the rows still unchosen ----------------
        const unsigned zm = sl.zm;
        int rq[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) rq[q] = (q < kb) ? lrow[c0 + q] : 0;
        const int S = nthr / nr;                         // threads per row
        const int s = tid / nr, r = tid - s * nr;
        if (s < S && ord[r] < 0) {
            T mr[KB];
            gepp_vload(W + static_cast<size_t>(r) * ws + c0, mr);
            if (kb == KB && zm == 0)
                gepp_rank_row<T, true, QB>(W, ws, r, s, S, j0, w, mr, W, ws, rq, kb, zm);
            else
                gepp_rank_row<T, false, QB>(W, ws, r, s, S, j0, w, mr, W, ws, rq, kb, zm);
        }
        __syncthreads();
    }
}

// The same selection with a lookahead inside the node, for a CTA of at
// least 2 x 256 threads and nr <= 256 rows.  The first warps own the rows
// (one per thread, as above); warps 8.. form the update group, thread u of
// which also works on row u.  Per panel p (columns [c0, c0 + kb)):
//   row warps     the column chain of panel p on the slab they updated
//                 last; then the pivot rows' trailing columns (the
//                 triangle); then panel p's rank-KB update of their own rows
//                 on the next slab [j0, j0 + KB) only;
//   update warps  meanwhile, panel p-1's rank-KB update of every row not
//                 chosen by then, on the columns after that slab.
// Two block barriers per panel order the phases: every element still takes
// its pivots' updates in ascending order (the near slab of panel p after the
// far part of panel p-1 has reached it), each multiplier is one IEEE
// division, so rows, multipliers and factors are node_gepp_blocked's bit
// for bit.  Named barrier 1 is used among the row warps.
// End of the near slab after column j0: KB columns, rounded up to a 16-byte
// chunk so that the row warps' near update and the update warps' far update
// (which run at the same time, each rewriting whole chunks) never share a
// chunk.
__device__ __forceinline__ int near_end(int j0, int w) { return min((j0 + kGeppKB + 3) & ~3, w); }

template <typename T>
__device__ void node_gepp_la(T* W, int ws, int nr, int w, int ns, const int* ids, int* ord, int* winp, int* lrow,
                             GeppSlots<T>& sl, unsigned* zmp, int* zero_first) {
    constexpr int KB = kGeppKB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwo = (nr + 31) >> 5;                   // row warps
    const bool rowgrp = warp < nwo;
    const bool updgrp = tid >= 256;
    const int u = tid - 256;                           // update-group row
    const bool own = tid < nr;
    T* const wr = W + static_cast<size_t>(own ? tid : 0) * ws;
    bool live = own && ord[tid] < 0;
    const int myid = own ? ids[tid] : INT_MAX;
    if (ns <= 0) {
        __syncthreads();
        return;
    }
    const int npan = (ns + KB - 1) / KB;
    T P[KB];                                           // row warps: the panel's values, then multipliers
    for (int p = 0; p <= npan; ++p) {
        const int c0 = p * KB;
        const int kb = p < npan ? min(KB, ns - c0) : 0;
        const int j0 = c0 + kb;
        // ---------------- update warps: panel p-1, far columns ----------------
        if (updgrp && p >= 1 && u < nr) {
            const int pc0 = (p - 1) * KB;
            const int pkb = min(KB, ns - pc0);
            const int far0 = near_end(pc0 + pkb, w);  // after the slab the row warps updated
            const int o = ord[u];                       // -1, or a step of panel p or later: still to update
            if (far0 < w && (o < 0 || o >= pc0 + KB)) {
                const unsigned pzm = zmp[(p - 1) & 1];
                int prq[KB];
#pragma unroll
                for (int q = 0; q < KB; ++q) prq[q] = (q < pkb) ? lrow[pc0 + q] : 0;
                T mr[KB];
                gepp_vload(W + static_cast<size_t>(u) * ws + pc0, mr);
                if (pkb == KB && pzm == 0)
                    gepp_rank_row<T, true>(W, ws, u, 0, 1, far0, w, mr, W, ws, prq, pkb, pzm);
                else
                    gepp_rank_row<T, false>(W, ws, u, 0, 1, far0, w, mr, W, ws, prq, pkb, pzm);
            }
        }
        int rq[KB];
        unsigned zm = 0;
        // ---------------- row warps: column chain of panel p ----------------
        if (p < npan && rowgrp) {
            if (own) {
                gepp_vload(wr + c0, P);
            } else {
#pragma unroll
                for (int k = 0; k < KB; ++k) P[k] = T(0);
            }
            int khi;
            unsigned klo;
            gepp_key(P[0], live, khi, klo);
            int chosen = -1;
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                rq[k] = 0;
                if (k < kb) {
                    const int c = c0 + k;
                    const int buf = c & 1;
                    int mhi;
                    unsigned mlo;
                    const int wl = gepp_warp_best<T>(khi, klo, lane, mhi, mlo);
                    if (lane == wl) {
                        sl.key[buf][warp] = mhi;
                        sl.key_lo[buf][warp] = mlo;
                        sl.row[buf][warp] = tid;
                        gepp_vstore(&sl.val[buf][warp][0], P);
                    }
                    gepp_bar(1, nwo * 32);
                    const int phi = lane < nwo ? sl.key[buf][lane] : -1;
                    const unsigned plo = lane < nwo ? sl.key_lo[buf][lane] : 0u;
                    const int prow = lane < nwo ? sl.row[buf][lane] : INT_MAX;
                    const int ghi = __reduce_max_sync(0xffffffffu, phi);
                    bool cand = (phi == ghi);
                    if (sizeof(T) == 8) {
                        const unsigned glo = __reduce_max_sync(0xffffffffu, cand ? plo : 0u);
                        cand = cand && (plo == glo);
                    }
                    const int lr = __reduce_min_sync(0xffffffffu, cand ? prow : INT_MAX);
                    T U[KB];
                    gepp_vload(&sl.val[buf][lr >> 5][0], U);
                    rq[k] = lr;
                    const T pv = U[k];
                    const bool pz = (pv == T(0));
                    if (pz) zm |= 1u << k;
                    const bool win = live && (tid == lr);
                    if (win) chosen = k;
                    const bool upd = live && !win && !pz;
                    const T l = P[k] / (upd ? pv : T(1));
                    if (upd) P[k] = l;
#pragma unroll
                    for (int j = k + 1; j < KB; ++j)
                        if (j < kb && upd) P[j] = fma(-l, U[j], P[j]);
                    live = live && !win;
                    gepp_key(P[(k + 1) < KB ? k + 1 : KB - 1], live && k + 1 < kb, khi, klo);
                }
            }
            if (chosen >= 0) {
                ord[tid] = c0 + chosen;
                winp[c0 + chosen] = myid;
                lrow[c0 + chosen] = tid;
            }
            if (chosen >= 0 || live) gepp_store_panel(wr + c0, P, kb);
            if (tid == 0) {
                zmp[p & 1] = zm;
                if (zero_first != nullptr && zm != 0 && *zero_first < 0) *zero_first = c0 + __ffs(zm) - 1;
            }
        }
        __syncthreads();
        if (p == npan) break;
        // ---------------- row warps: triangle of panel p (the pivot rows'
        // multipliers are in W since the chain stored them) ----------------
        if (rowgrp && kb > 1) {
            for (int j = j0 + tid; j < w; j += nwo * 32) {
                T uu[KB];
#pragma unroll
                for (int q = 0; q < KB; ++q) uu[q] = (q < kb) ? W[static_cast<size_t>(rq[q]) * ws + j] : T(0);
#pragma unroll
                for (int q = 1; q < KB; ++q) {
                    if (q < kb) {
#pragma unroll
                        for (int qq = 0; qq < KB; ++qq)
                            if (qq < q && !((zm >> qq) & 1u))
                                uu[q] = fma(-W[static_cast<size_t>(rq[q]) * ws + c0 + qq], uu[qq], uu[q]);
                    }
                }
#pragma unroll
                for (int q = 1; q < KB; ++q)
                    if (q < kb) W[static_cast<size_t>(rq[q]) * ws + j] = uu[q];
            }
        }
        __syncthreads();
        // ---------------- row warps: panel p on the next slab ----------------
        if (rowgrp && live && j0 < w) {
            const int jn = near_end(j0, w);
            if (kb == KB && zm == 0)
                gepp_rank_row<T, true>(W, ws, tid, 0, 1, j0, jn, P, W, ws, rq, kb, zm);
            else
                gepp_rank_row<T, false>(W, ws, tid, 0, 1, j0, jn, P, W, ws, rq, kb, zm);
        }
    }
    __syncthreads();
}

}  // namespace lu
