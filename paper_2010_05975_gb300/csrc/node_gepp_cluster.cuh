// Blocked GEPP for a tournament node spread over a thread-block cluster (the
// local LUP of TournPivot, Section 7.3, when the node's rows exceed one SM).
// CTA rank q holds node rows [q*R, q*R + nloc) (nloc <= 32), the node's rows
// being in ascending position order across the cluster.
//
// Per column step, warp 0 of every CTA (one lane per row) finds the CTA's
// candidate by warp reductions and stores its key and KB panel values into
// every CTA's candidate table (remote shared-memory stores); one cluster
// barrier (every thread of every CTA) makes them visible, and each CTA then
// folds the C candidates from its own shared memory and updates its rows'
// panel values in registers.  Per KB-column panel: one more cluster
// barrier, after which every CTA gathers the panel's pivot rows (from their
// owners, through distributed shared memory) into a local buffer, finishes
// their trailing columns (triangle) and applies the rank-KB update to its
// own unchosen rows.  The per-element operations and their order are those
// of the column-by-column GEPP (see node_gepp.cuh), so the result is the
// same bit for bit.  There is no spin-wait: every synchronization is a
// hardware cluster barrier.
#pragma once
#include "node_gepp.cuh"
#include <cooperative_groups.h>

namespace lu {

// One CTA's candidate of a column step.
template <typename T>
struct GeppCand {
    int key;
    unsigned key_lo;
    int row;                                // node row
    int pos;                                // row position
    alignas(16) T val[kGeppKB];             // its panel values
};

template <typename T>
struct GeppClusterSlot {
    GeppCand<T> cand[2][16];                // [step parity][CTA rank], written by the CTAs
    int gk[kGeppKB];                        // the panel's pivot rows (node rows)
    int gk_prev[kGeppKB];                   // the previous panel's
    unsigned zm;                            // the panel's zero-pivot steps
};

// GEPP on the node's rows, columns [0, ns) of the w-column panel.
//   W, ws   this CTA's nloc rows (stride gepp_ws<T>(w), 16-byte aligned);
//           on return as for node_gepp_blocked, except that with
//           writeback false the chosen rows' columns after their panel are
//           not finished (only the root needs them).
//   R, C, q rows per CTA, CTAs in the cluster, this CTA's rank.
//   ids     positions of this CTA's rows; ord[r] = -1 on entry, on return
//           the step that chose local row r, or -1.
//   winp    winp[c] = position of the step-c pivot row (every CTA).
//   Ub      local buffer of kGeppKB rows, stride ws.
//   zero_first  (may be null) set to the first step with a zero pivot when < 0.
// Requires blockDim.x >= 32 (a multiple of 32), nloc <= 32, R <= 32, C <= 16.
// Called by every thread of every CTA of the cluster with the same w, ns,
// R and C; uses cluster barriers.
template <typename T>
__device__ void node_gepp_cluster(T* W, int ws, int nloc, int R, int C, int q, int w, int ns, const int* ids,
                                  int* ord, int* winp, T* Ub, GeppClusterSlot<T>& sl, int* zero_first,
                                  bool writeback) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int KB = kGeppKB;
    constexpr int V = 16 / sizeof(T);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const bool own = (warp == 0) && lane < nloc;
    T* const wr = W + static_cast<size_t>(own ? lane : 0) * ws;
    bool live = own && ord[lane] < 0;
    const int myid = own ? ids[lane] : INT_MAX;
    const int grow = q * R + lane;
    int prev_j0 = -1, prev_kb = 0;                      // the previous panel, when its rows need writing back
    for (int c0 = 0; c0 < ns; c0 += KB) {
        const int kb = min(KB, ns - c0);
        const int j0 = c0 + kb;
        // ---------------- column steps (warp 0 holds the rows; every warp takes the barriers) ----------------
        T P[KB];
        int khi = -1;
        unsigned klo = 0u;
        unsigned zm = 0;
        int chosen = -1;
        int gk[KB];
        if (warp == 0) {
            if (own) {
                gepp_vload(wr + c0, P);
            } else {
#pragma unroll
                for (int k = 0; k < KB; ++k) P[k] = T(0);
            }
            gepp_key(P[0], live, khi, klo);
        }
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            gk[k] = 0;
            if (k < kb) {
                const int c = c0 + k;
                const int buf = c & 1;
                if (warp == 0) {
                    int mhi;
                    unsigned mlo;
                    const int wl = gepp_warp_best<T>(khi, klo, lane, mhi, mlo);
                    const int crow = __shfl_sync(0xffffffffu, grow, wl);
                    const int cpos = __shfl_sync(0xffffffffu, myid, wl);
                    T cv[KB];
#pragma unroll
                    for (int j = 0; j < KB; ++j) cv[j] = __shfl_sync(0xffffffffu, P[j], wl);
                    if (lane < C) {
                        // this CTA's candidate into CTA lane's table
                        GeppCand<T>* dst = &cluster.map_shared_rank(&sl, lane)->cand[buf][q];
                        *reinterpret_cast<int4*>(dst) = make_int4(mhi, static_cast<int>(mlo), crow, cpos);
                        gepp_vstore(&dst->val[0], cv);
                    }
                }
                cluster.sync();
                if (warp == 0) {
                    const GeppCand<T>* tab = &sl.cand[buf][0];
                    const int phi = lane < C ? tab[lane].key : -1;
                    const unsigned plo = lane < C ? static_cast<unsigned>(tab[lane].key_lo) : 0u;
                    const int prow = lane < C ? tab[lane].row : INT_MAX;
                    const int ghi = __reduce_max_sync(0xffffffffu, phi);
                    bool cand = (phi == ghi);
                    if (sizeof(T) == 8) {
                        const unsigned glo = __reduce_max_sync(0xffffffffu, cand ? plo : 0u);
                        cand = cand && (plo == glo);
                    }
                    const int g = __reduce_min_sync(0xffffffffu, cand ? prow : INT_MAX);
                    const int src = min(max(g / R, 0), C - 1);
                    T U[KB];
                    gepp_vload(&tab[src].val[0], U);
                    if (lane == 0) winp[c] = tab[src].pos;
                    gk[k] = g;
                    const T pv = U[k];
                    const bool pz = (pv == T(0));
                    if (pz) zm |= 1u << k;
                    const bool win = live && (grow == g);
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
        }
        if (warp == 0) {
            if (chosen >= 0) ord[lane] = c0 + chosen;
            if (chosen >= 0 || live) gepp_store_panel(wr + c0, P, kb);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < KB; ++k) sl.gk[k] = gk[k];
                sl.zm = zm;
                if (zero_first != nullptr && zm != 0 && *zero_first < 0) *zero_first = c0 + __ffs(zm) - 1;
            }
        }
        // the panel's pivot rows are in their owners' W; every rank-KB update before is done
        cluster.sync();
        if (writeback && prev_j0 >= 0) {
            // the previous panel's pivot rows held here take their finished trailing columns
            for (int e = tid; e < prev_kb * (w - prev_j0); e += nthr) {
                const int qq = e / (w - prev_j0), j = prev_j0 + e % (w - prev_j0);
                const int g = sl.gk_prev[qq];
                if (g >= q * R && g < q * R + nloc)
                    W[static_cast<size_t>(g - q * R) * ws + j] = Ub[static_cast<size_t>(qq) * ws + j];
            }
            prev_j0 = -1;
            __syncthreads();
        }
        if (j0 >= w) continue;
        zm = sl.zm;                                       // every thread: the panel's zero-pivot steps
        // gather the pivot rows' columns [c0, w) into Ub
        const int nch = (w - c0 + V - 1) / V;
        for (int e = tid; e < kb * nch; e += nthr) {
            const int qq = e / nch, i = e % nch;
            const int g = sl.gk[qq];
            const int owner = min(max(g / R, 0), C - 1);
            const int lr = min(max(g - owner * R, 0), R - 1);
            const T* srow = cluster.map_shared_rank(W, owner) + static_cast<size_t>(lr) * ws;
            T x[V];
            gepp_ld16(srow + c0 + V * i, x);
            gepp_st16(Ub + static_cast<size_t>(qq) * ws + c0 + V * i, x);
        }
        __syncthreads();
        // triangle: the pivot rows' trailing columns, in pivot order
        if (kb > 1) {
            for (int j = j0 + tid; j < w; j += nthr) {
                T u[KB];
#pragma unroll
                for (int qq = 0; qq < KB; ++qq) u[qq] = (qq < kb) ? Ub[static_cast<size_t>(qq) * ws + j] : T(0);
#pragma unroll
                for (int qv = 1; qv < KB; ++qv) {
                    if (qv < kb) {
#pragma unroll
                        for (int qq = 0; qq < KB; ++qq)
                            if (qq < qv && !((zm >> qq) & 1u))
                                u[qv] = fma(-Ub[static_cast<size_t>(qv) * ws + c0 + qq], u[qq], u[qv]);
                    }
                }
#pragma unroll
                for (int qv = 1; qv < KB; ++qv)
                    if (qv < kb) Ub[static_cast<size_t>(qv) * ws + j] = u[qv];
            }
            __syncthreads();
        }
        // rank-KB update of this CTA's unchosen rows
        {
            int rq[KB];
#pragma unroll
            for (int qq = 0; qq < KB; ++qq) rq[qq] = qq;
            const int S = nloc > 0 ? nthr / nloc : 0;
            const int s = nloc > 0 ? tid / nloc : 1, r = tid - s * nloc;
            if (s < S && ord[r] < 0) {
                T mr[KB];
                gepp_vload(W + static_cast<size_t>(r) * ws + c0, mr);
                if (kb == KB && zm == 0)
                    gepp_rank_row<T, true>(W, ws, r, s, S, j0, w, mr, Ub, ws, rq, kb, zm);
                else
                    gepp_rank_row<T, false>(W, ws, r, s, S, j0, w, mr, Ub, ws, rq, kb, zm);
            }
        }
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < KB; ++k) sl.gk_prev[k] = sl.gk[k];
        }
        prev_j0 = j0;
        prev_kb = kb;
        __syncthreads();
    }
    if (writeback && prev_j0 >= 0) {
        cluster.sync();
        for (int e = tid; e < prev_kb * (w - prev_j0); e += nthr) {
            const int qq = e / (w - prev_j0), j = prev_j0 + e % (w - prev_j0);
            const int g = sl.gk_prev[qq];
            if (g >= q * R && g < q * R + nloc)
                W[static_cast<size_t>(g - q * R) * ws + j] = Ub[static_cast<size_t>(qq) * ws + j];
        }
    }
    __syncthreads();
}

}  // namespace lu
