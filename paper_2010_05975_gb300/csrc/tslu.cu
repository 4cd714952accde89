// Tournament pivoting (TournPivot, Section 7.3) and pivot application for
// the binary64 factorization.
//
// One launch per tree level.  A node is handled by one thread-block cluster
// of C CTAs; each CTA holds up to R of the node's candidate rows (their
// current panel values) in shared memory.  A GEPP column step is
//   local argmax  ->  one cluster barrier  ->  every CTA reads the C local
//   winners and the pivot row through distributed shared memory  ->  local
//   rank-1 update of its unchosen rows.
// The arithmetic per element is the oracle's: multiplier = a / pivot (IEEE
// division), update a = fma(-l, u, a) in ascending pivot order; ties in |a|
// go to the smallest row position.  Because a node's choice does not depend
// on the order its candidates are stacked in, the first tree levels, whose
// nodes keep all their rows, are skipped: the first launched level takes
// contiguous row ranges of H rows.
#include "common.cuh"
#include "node_gepp.cuh"
#include "node_gepp_cluster.cuh"
#include "prof.cuh"
#include <cooperative_groups.h>
#include <climits>

namespace cg = cooperative_groups;

namespace lu {

TsluShape tslu_shape(int m, int k, int w, int h, int max_cluster, int elem) {
    TsluShape s{};
    const int nact = m - k;
    int H = h;
    if (h <= w) {
        H = h;
        while (H <= w) H *= 2;
    }
    s.H = H;
    s.nsuper = cdiv(nact, H);
    s.nr_max = (s.nsuper == 1) ? nact : (H > 2 * w ? H : 2 * w);
    // binary64: spread the node over up to max_cluster CTAs (the DFMA pipe,
    // about 2 FMA/clk/SM, bounds each CTA's update); binary32: the fewest CTAs
    // whose rows fit in shared memory (the cluster barrier per column is then
    // the cost to avoid).
    const long long budget = (elem == 8) ? 32768 : 200 * 1024;
    int C = 1, R = s.nr_max;
    while (C < max_cluster && static_cast<long long>(R) * (w + 1) * elem > budget) {
        C *= 2;
        R = cdiv(s.nr_max, C);
    }
    s.C = C;
    s.R = R;
    auto bytes = [&](int ws) {
        return static_cast<size_t>(R) * ws * elem + static_cast<size_t>(w) * elem +
               static_cast<size_t>(R) * 2 * sizeof(int) + static_cast<size_t>(2 * w) * sizeof(int);
    };
    // A node on one CTA whose rows fit one per thread runs the blocked GEPP
    // (mode 1); a node over a cluster of at most 32 rows per CTA, the
    // cluster-blocked GEPP (mode 2); anything else, the column-by-column
    // GEPP over the cluster (mode 0).
    const int threads = (elem == 4) ? 512 : kTsluThreads;
    const int bws = (elem == 8) ? gepp_ws<double>(w) : gepp_ws<float>(w);
    s.blocked = 0;
    s.ws = w + 1;
    if (C == 1 && R <= threads && bytes(bws) <= kTsluSmemLimit) {
        s.blocked = 1;
        s.ws = bws;
    } else {
        int C2 = 2;
        while (C2 < max_cluster && cdiv(s.nr_max, C2) > 32) C2 *= 2;
        const int R2 = cdiv(s.nr_max, C2);
        const size_t b2 = static_cast<size_t>(R2 + kGeppKB) * bws * elem + static_cast<size_t>(w) * elem +
                          static_cast<size_t>(R2) * 2 * sizeof(int) + static_cast<size_t>(2 * w) * sizeof(int);
        // (the candidates' positions are sorted in W's space before the rows arrive)
        const bool sort_fits = static_cast<size_t>(R2) * bws * elem >= static_cast<size_t>(s.nr_max) * sizeof(int);
        if (R2 <= 32 && b2 <= kTsluSmemLimit && sort_fits) {
            s.blocked = 2;
            s.C = C2;
            s.R = R2;
            s.ws = bws;
            s.smem = b2;
            return s;
        }
    }
    s.smem = bytes(s.ws);
    return s;
}

template <typename T>
struct LevelArgs {
    const T* A;
    int lda, m, k, w, H;
    int level;          // 0: first launched level (contiguous row ranges)
    int nnode;          // nodes at this level
    int nchild;         // nodes at the level below (level > 0)
    int root;           // this level is the root (one node)
    const int* child_list;
    const int* child_cnt;
    int* out_list;      // node-major, stride w
    int* out_cnt;
    T* a00;             // root: w x w rows of the factored winners, pivot order
    int* info;          // root: first zero pivot
    int C, R;
    int ws;             // row stride of W
    int blocked;        // GEPP mode: 1 one-CTA blocked, 2 cluster-blocked, 0 column by column
};

template <typename T>
__device__ __forceinline__ bool better(T v1, int p1, T v2, int p2) {
    return v1 > v2 || (v1 == v2 && p1 < p2);
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& p, int& l) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        T ov = __shfl_down_sync(0xffffffffu, v, off);
        int op = __shfl_down_sync(0xffffffffu, p, off);
        int ol = __shfl_down_sync(0xffffffffu, l, off);
        if (better(ov, op, v, p)) {
            v = ov;
            p = op;
            l = ol;
        }
    }
}

template <typename T>
constexpr int tslu_threads() { return sizeof(T) == 4 ? 512 : kTsluThreads; }

// What changes from one tree level to the next (the rest is in LevelArgs).
struct LevelView {
    int level, nchild, root;
    const int* child_list;
    const int* child_cnt;
    int* out_list;
    int* out_cnt;
};

// One node of one tree level (the CTA, or cluster of a.C CTAs, that runs
// it).  MODE 1: one-CTA nodes, blocked GEPP; MODE 2: nodes over a cluster,
// cluster-blocked GEPP; MODE 0: nodes over a cluster, column-by-column GEPP.
// Child lists and counts are read through L2 (in the one-launch tree they
// were written by other CTAs of the same launch).  Ends with a block (or
// cluster) barrier.
template <typename T, int MODE, bool LA_ONLY = false>
__device__ __forceinline__ void tslu_node(const LevelArgs<T>& a, const LevelView& v, int node) {
    cg::cluster_group cluster = cg::this_cluster();
    const int q = static_cast<int>(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarp = blockDim.x >> 5;
    const int w = a.w, ws = a.ws;

    int nr, r0 = 0, cl = 0;
    const int* lp = nullptr;
    const int* rp = nullptr;
    if (v.level == 0) {
        r0 = a.k + node * a.H;
        nr = min(a.H, a.m - r0);
    } else {
        const int left = 2 * node, right = 2 * node + 1;
        cl = __ldcg(v.child_cnt + left);
        lp = v.child_list + static_cast<size_t>(left) * w;
        if (right >= v.nchild) {            // odd last node goes up unchanged
            if (q == 0) {
                for (int i = tid; i < cl; i += blockDim.x) v.out_list[static_cast<size_t>(node) * w + i] = __ldcg(lp + i);
                if (tid == 0) v.out_cnt[node] = cl;
            }
            return;
        }
        rp = v.child_list + static_cast<size_t>(right) * w;
        nr = cl + __ldcg(v.child_cnt + right);
    }
    if (!(v.root || nr > w)) {              // a node that keeps all its rows
        if (q == 0) {
            for (int i = tid; i < nr; i += blockDim.x) v.out_list[static_cast<size_t>(node) * w + i] = r0 + i;
            if (tid == 0) v.out_cnt[node] = nr;
        }
        return;
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* W = reinterpret_cast<T*>(smem_raw);              // R x ws
    T* Ub = W + static_cast<size_t>(a.R) * ws;           // MODE 2: kGeppKB x ws
    T* prow = Ub + (MODE == 2 ? static_cast<size_t>(kGeppKB) * ws : 0);   // w
    int* ids = reinterpret_cast<int*>(prow + w);          // R
    int* ord = ids + a.R;                                 // R
    int* winp = ord + a.R;                                // w
    int* lrow = winp + w;                                 // w (blocked GEPP)
    __shared__ T slot_v[2];
    __shared__ int slot_p[2], slot_l[2];
    __shared__ T part_v[2][32];
    __shared__ int part_p[2][32], part_l[2][32];
    __shared__ int s_owner, s_lr, s_zero;

    const int i0 = q * a.R;
    const int nloc = max(0, min(a.R, nr - i0));
    if (MODE != 0 && v.level > 0) {
        // The blocked GEPPs break ties by row: stack the candidates in
        // ascending position order (the selection does not depend on it);
        // this CTA keeps ranks [i0, i0 + nloc).
        int* tmp = reinterpret_cast<int*>(W);             // nr positions, before the rows arrive
        for (int i = tid; i < nr; i += blockDim.x) tmp[i] = (i < cl) ? __ldcg(lp + i) : __ldcg(rp + i - cl);
        __syncthreads();
        for (int i = tid; i < nr; i += blockDim.x) {
            const int pi = tmp[i];
            int rank = 0;
            for (int j = 0; j < nr; ++j) rank += (tmp[j] < pi) ? 1 : 0;
            if (rank >= i0 && rank < i0 + nloc) ids[rank - i0] = pi;
        }
        __syncthreads();
    }
    for (int r = warp; r < nloc; r += nwarp) {
        const int gi = i0 + r;
        const int pos = (v.level == 0) ? (r0 + gi) : (MODE != 0) ? ids[r] : (gi < cl ? __ldcg(lp + gi) : __ldcg(rp + gi - cl));
        if (lane == 0) {
            ids[r] = pos;
            ord[r] = -1;
        }
        const T* src = a.A + idx(pos, a.k, a.lda);
        for (int j = lane; j < w; j += 32) W[r * ws + j] = src[j];
    }
    if (tid == 0) s_zero = -1;
    __syncthreads();

    const int ns = min(nr, w);
    if constexpr (MODE == 1) {
        __shared__ GeppSlots<T> gslots;
        if (LA_ONLY || (sizeof(T) == 4 && blockDim.x >= 512 && nloc <= 256)) {
            // binary32 nodes: the update warps run one panel behind the row warps
            __shared__ unsigned s_zmp[2];
            node_gepp_la<T>(W, ws, nloc, w, ns, ids, ord, winp, lrow, gslots, s_zmp, &s_zero);
        } else {
            node_gepp_blocked<T>(W, ws, nloc, w, ns, ids, ord, winp, lrow, gslots, &s_zero);
        }
    } else if constexpr (MODE == 2) {
        __shared__ GeppClusterSlot<T> cslot;
        node_gepp_cluster<T>(W, ws, nloc, a.R, a.C, q, w, ns, ids, ord, winp, Ub, cslot, q == 0 ? &s_zero : nullptr,
                             v.root != 0);
    } else {
        // Row groups: tpr (a power of two <= 32) threads per row, all in one warp.
        int tpr = 1;
        while (tpr < 32 && 2 * tpr * max(nloc, 1) <= static_cast<int>(blockDim.x)) tpr *= 2;
        const int rows_per_pass = static_cast<int>(blockDim.x) / tpr;
        const int jj = tid % tpr;
        const unsigned gmask = (tpr == 32) ? 0xffffffffu : (((1u << tpr) - 1u) << (lane & ~(tpr - 1)));
        const int glead = lane & ~(tpr - 1);

        // candidate of column 0 (later columns come out of the fused update)
        T bv = T(-1);
        int bp = INT_MAX, bl = -1;
        if (jj == 0 && ns > 0)
            for (int r = tid / tpr; r < nloc; r += rows_per_pass) {
                T v = abs(W[r * ws + 0]);
                if (!(v == v)) v = T(INFINITY);     // a NaN row still wins: the step always has a pivot row
                if (better(v, ids[r], bv, bp)) {
                    bv = v;
                    bp = ids[r];
                    bl = r;
                }
            }
        for (int c = 0; c < ns; ++c) {
            // 1. per-warp argmax of the candidates for column c (double-buffered
            //    partials: a warp may run one step ahead of a slow reader)
            const int buf = c & 1;
            warp_argmax(bv, bp, bl);
            if (lane == 0) {
                part_v[buf][warp] = bv;
                part_p[buf][warp] = bp;
                part_l[buf][warp] = bl;
            }
            __syncthreads();
            int lr, owner;
            if (a.C == 1) {
                // one-CTA node: every thread folds the partials itself
                T v = part_v[buf][0];
                int p = part_p[buf][0], l = part_l[buf][0];
                for (int i = 1; i < nwarp; ++i)
                    if (better(part_v[buf][i], part_p[buf][i], v, p)) {
                        v = part_v[buf][i];
                        p = part_p[buf][i];
                        l = part_l[buf][i];
                    }
                lr = l;
                owner = 0;
                if (tid == 0) winp[c] = p;
            } else {
                if (warp == 0) {
                    bv = lane < nwarp ? part_v[buf][lane] : T(-1);
                    bp = lane < nwarp ? part_p[buf][lane] : INT_MAX;
                    bl = lane < nwarp ? part_l[buf][lane] : -1;
                    warp_argmax(bv, bp, bl);
                    if (lane == 0) {
                        slot_v[buf] = bv;
                        slot_p[buf] = bp;
                        slot_l[buf] = bl;
                    }
                }
                cluster.sync();
                // 2. cluster-wide winner, identical in every CTA
                if (warp == 0) {
                    T v = T(-1);
                    int p = INT_MAX, l = -1;
                    if (lane < a.C) {
                        v = cluster.map_shared_rank(slot_v, lane)[buf];
                        p = cluster.map_shared_rank(slot_p, lane)[buf];
                        l = cluster.map_shared_rank(slot_l, lane)[buf];
                    }
                    int o = (lane < a.C) ? lane : -1;
    #pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        T ov = __shfl_down_sync(0xffffffffu, v, off);
                        int op = __shfl_down_sync(0xffffffffu, p, off);
                        int ol = __shfl_down_sync(0xffffffffu, l, off);
                        int oo = __shfl_down_sync(0xffffffffu, o, off);
                        if (better(ov, op, v, p)) {
                            v = ov;
                            p = op;
                            l = ol;
                            o = oo;
                        }
                    }
                    if (lane == 0) {
                        s_owner = o;
                        s_lr = l;
                        winp[c] = p;
                        if (o == q) ord[l] = c;
                    }
                }
                __syncthreads();
                owner = s_owner;
                lr = s_lr;
            }
            // 3. the pivot row (never written again): in place for a one-CTA node,
            //    else copied from the owner's shared memory
            const T* pr;
            if (a.C == 1) {
                pr = W + lr * ws;
            } else {
                const T* rW = cluster.map_shared_rank(W, owner);
                for (int j = c + tid; j < w; j += blockDim.x) prow[j] = rW[lr * ws + j];
                __syncthreads();
                pr = prow;
            }
            const T pv = pr[c];
            if (pv == T(0) && tid == 0 && s_zero < 0) s_zero = c;
            // 4. fused: multiplier (one division per row, shuffled to the row's
            //    threads), rank-1 update, and the candidate for column c+1.
            bv = T(-1);
            bp = INT_MAX;
            bl = -1;
            const bool next = (c + 1 < ns);
            for (int r = tid / tpr; r < nloc; r += rows_per_pass) {
                if (a.C == 1 && r == lr) {                       // chosen now: mark it, leave it
                    if (jj == 0) ord[r] = c;
                    continue;
                }
                if (ord[r] >= 0) continue;                       // uniform over the row's threads
                T* wr = W + r * ws;
                if (pv != T(0)) {
                    T l = T(0);
                    if (jj == 0) l = wr[c] / pv;
                    l = __shfl_sync(gmask, l, glead);
                    if (jj == 0) wr[c] = l;
                    for (int j = c + 1 + jj; j < w; j += tpr) wr[j] = fma(-l, pr[j], wr[j]);
                }
                if (next && jj == 0) {
                    T v = abs(wr[c + 1]);
                    if (!(v == v)) v = T(INFINITY);
                    if (better(v, ids[r], bv, bp)) {
                        bv = v;
                        bp = ids[r];
                        bl = r;
                    }
                }
            }
        }
    }
    __syncthreads();

    if (q == 0) {
        for (int i = tid; i < ns; i += blockDim.x) v.out_list[static_cast<size_t>(node) * w + i] = winp[i];
        if (tid == 0) v.out_cnt[node] = ns;
    }
    if (v.root) {
        for (int r = warp; r < nloc; r += nwarp) {
            const int o = ord[r];
            if (o < 0) continue;
            for (int j = lane; j < w; j += 32) a.a00[static_cast<size_t>(o) * w + j] = W[r * ws + j];
        }
        if (q == 0 && tid == 0 && s_zero >= 0 && *a.info == 0) *a.info = a.k + s_zero + 1;
    }
    cluster.sync();     // no CTA leaves while another may still read its shared memory
}

// One tree level per launch: node = blockIdx.x / a.C.  Separate
// instantiations per mode, so that each keeps its own register allocation.
template <typename T, int MODE>
__global__ void __launch_bounds__(tslu_threads<T>()) tslu_level_kernel(const __grid_constant__ LevelArgs<T> a) {
    const LevelView v{a.level, a.nchild, a.root, a.child_list, a.child_cnt, a.out_list, a.out_cnt};
    tslu_node<T, MODE>(a, v, static_cast<int>(blockIdx.x) / a.C);
}

// The whole tree in one launch, for one-CTA nodes (MODE 1; binary32 nodes
// of at most 256 rows, which take the lookahead GEPP): CTA i runs leaf
// i, then climbs.  A node's two children end on different CTAs; the one
// that finishes second (an atomic count per parent node, `arrive`, zero at
// launch) goes on with the parent, the other exits, so no CTA ever waits
// for another.  A node without a sibling (the odd last one) passes its list
// up by itself.  Level L's nodes sit at list/count index base_L + node
// (base_0 = 0, base_{L+1} = base_L + nodes_L).  a describes level 0.
template <typename T>
__global__ void __launch_bounds__(tslu_threads<T>()) tslu_tree_kernel(const __grid_constant__ LevelArgs<T> a0,
                                                                      int* __restrict__ arrive) {
    __shared__ int s_go;
    int node = static_cast<int>(blockIdx.x), nn = a0.nnode, base = 0, pbase = 0, pnn = 0;
    for (int level = 0;; ++level) {
        const LevelView v{level, pnn, nn == 1 ? 1 : 0, a0.out_list + static_cast<size_t>(pbase) * a0.w,
                          a0.out_cnt + pbase, a0.out_list + static_cast<size_t>(base) * a0.w, a0.out_cnt + base};
        tslu_node<T, 1, sizeof(T) == 4>(a0, v, node);
        if (nn == 1) return;
        __threadfence();                                  // this node's list (and a00) before the count
        __syncthreads();
        if ((node ^ 1) < nn) {
            if (threadIdx.x == 0) {
                s_go = atomicAdd(arrive + base + nn + (node >> 1), 1);
                __threadfence();                          // the sibling's list after the count
            }
            __syncthreads();
            if (s_go == 0) return;                        // the sibling is still running: it goes on
        }
        pbase = base;
        pnn = nn;
        base += nn;
        nn = (nn + 1) >> 1;
        node >>= 1;
    }
}

template <typename T>
static int launch_level(const LevelArgs<T>& args, int nnode, int C, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nnode * C));
    cfg.blockDim = dim3(tslu_threads<T>());
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope ps(LU_PROF_TSLU, s);
    if (args.blocked == 1)
        LU_TRY(cudaLaunchKernelEx(&cfg, tslu_level_kernel<T, 1>, args));
    else if (args.blocked == 2)
        LU_TRY(cudaLaunchKernelEx(&cfg, tslu_level_kernel<T, 2>, args));
    else
        LU_TRY(cudaLaunchKernelEx(&cfg, tslu_level_kernel<T, 0>, args));
    count_launches(1);
    return 0;
}

// Largest cluster the device runs for the tournament kernel: 16 where the
// non-portable size is available, else the portable 8.
int tslu_max_cluster() {
    static std::once_flag once;
    static int cached = kTsluMaxCluster;
    std::call_once(once, [] {
        int best = kTsluMaxCluster;
        if (cudaFuncSetAttribute(tslu_level_kernel<double, 0>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(tslu_level_kernel<float, 0>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(tslu_level_kernel<double, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(tslu_level_kernel<float, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
            // the largest binary64 node over 16 CTAs, in both cluster modes
            const TsluShape sh = tslu_shape(2 * kMaxPanel * 16, 0, kMaxPanel, 128, 16, sizeof(double));
            auto fits16 = [&](auto kernel) {
                if (smem_attr(kernel, sh.smem) != 0) return false;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(16);
                cfg.blockDim = dim3(kTsluThreads);
                cfg.dynamicSmemBytes = sh.smem;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 16;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int nclusters = 0;
                return cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0;
            };
            if (fits16(tslu_level_kernel<double, 0>) && fits16(tslu_level_kernel<double, 2>)) best = 16;
        }
        cudaGetLastError();
        cached = best;
    });
    return cached;
}

template <typename T>
int tslu_select(const T* A, int lda, int m, int k, int w, int h, int* lists, int* counts,
                size_t list_stride_nodes, T* a00, int* info, const int** root_list, cudaStream_t s) {
    const TsluShape sh = tslu_shape(m, k, w, h, tslu_max_cluster(), sizeof(T));
    if (int rc_ = sh.blocked == 1   ? smem_attr(tslu_level_kernel<T, 1>, sh.smem)
                  : sh.blocked == 2 ? smem_attr(tslu_level_kernel<T, 2>, sh.smem)
                                    : smem_attr(tslu_level_kernel<T, 0>, sh.smem))
        return rc_;
    int* list_buf[2] = {lists, lists + list_stride_nodes * w};
    int* cnt_buf[2] = {counts, counts + list_stride_nodes};
    LevelArgs<T> args{};
    args.A = A;
    args.lda = lda;
    args.m = m;
    args.k = k;
    args.w = w;
    args.H = sh.H;
    args.a00 = a00;
    args.info = info;
    args.C = sh.C;
    args.R = sh.R;
    args.ws = sh.ws;
    args.blocked = sh.blocked;

    int nn = sh.nsuper, cur = 0;
    args.level = 0;
    args.nnode = nn;
    args.nchild = 0;
    args.root = (nn == 1);
    args.child_list = nullptr;
    args.child_cnt = nullptr;
    // (binary32 nodes must fit the lookahead GEPP: rows <= 256 on 512 threads)
    if (sh.blocked == 1 && sh.C == 1 && (sizeof(T) == 8 || (sh.R <= 256 && tslu_threads<T>() >= 512))) {
        // the whole tree in one launch: lists and counts level after level,
        // arrival counts after the counts (2 list_stride_nodes each)
        args.out_list = lists;
        args.out_cnt = counts;
        int* arrive = counts + 2 * list_stride_nodes;
        int total = 0, rbase = 0;
        for (int k = nn; ; k = (k + 1) >> 1) {
            rbase = total;
            total += k;
            if (k == 1) break;
        }
        LU_TRY(cudaMemsetAsync(arrive, 0, sizeof(int) * static_cast<size_t>(total), s));
        {
            ProfScope ps(LU_PROF_TSLU, s);
            if (int rc_ = smem_attr(tslu_tree_kernel<T>, sh.smem)) return rc_;
            tslu_tree_kernel<T><<<nn, tslu_threads<T>(), sh.smem, s>>>(args, arrive);
            count_launches(1);
        }
        LU_LAUNCHED();
        *root_list = lists + static_cast<size_t>(rbase) * w;
        return 0;
    }
    args.out_list = list_buf[cur];
    args.out_cnt = cnt_buf[cur];
    if (int rc = launch_level(args, nn, sh.C, sh.smem, s)) return rc;
    int lvl = 1;
    while (nn > 1) {
        const int npar = (nn + 1) / 2;
        args.level = lvl++;
        args.nnode = npar;
        args.nchild = nn;
        args.root = (npar == 1);
        args.child_list = list_buf[cur];
        args.child_cnt = cnt_buf[cur];
        args.out_list = list_buf[cur ^ 1];
        args.out_cnt = cnt_buf[cur ^ 1];
        if (int rc = launch_level(args, npar, sh.C, sh.smem, s)) return rc;
        cur ^= 1;
        nn = npar;
    }
    *root_list = list_buf[cur];
    return 0;
}

template int tslu_select<double>(const double*, int, int, int, int, int, int*, int*, size_t, double*, int*,
                                 const int**, cudaStream_t);
template int tslu_select<float>(const float*, int, int, int, int, int, int*, int*, size_t, float*, int*, const int**,
                                cudaStream_t);

// ---------------------------------------------------------------------------
// Pivot application.  The w winners go to rows k..k+w-1 by LAPACK-style
// sequential swaps; one thread replays the swaps on row identities to get
// piv[k..k+w) and the final source row of every touched position.
// Positions touched are the top block [k, k+w) ("top t" = position k+t) and
// the original positions of winners from below it ("slot s" = position
// win[s] when win[s] >= k+w).  A top-origin row can be pushed into a slot
// and be a winner later, so its location is tracked as either kind.
// mv holds [count, dst[2w], src[2w]].
// ---------------------------------------------------------------------------
__global__ void pivot_moves_kernel(const int* __restrict__ win, int k, int w, int* __restrict__ piv,
                                   int* __restrict__ mv) {
    __shared__ int cT[kMaxPanel];   // original row now at top t
    __shared__ int cO[kMaxPanel];   // original row now at slot s
    __shared__ int loc[kMaxPanel];  // where the row that started at top t is: t' >= 0 top, -(s+1) slot
    __shared__ int wn[kMaxPanel];
    const int top = k + w;
    for (int t = threadIdx.x; t < w; t += blockDim.x) {
        cT[t] = k + t;
        loc[t] = t;
        wn[t] = win[t];
        cO[t] = win[t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < w; ++j) {
            const int o = wn[j];
            int where;                              // location of winner j
            if (o >= top) where = -(j + 1);         // slot j is untouched before swap j
            else where = loc[o - k];
            const int p = (where >= 0) ? (k + where) : wn[-where - 1];
            piv[k + j] = p;
            if (p == k + j) continue;
            const int ra = cT[j];
            int rb;
            if (where >= 0) {
                rb = cT[where];
                cT[where] = ra;
            } else {
                rb = cO[-where - 1];
                cO[-where - 1] = ra;
            }
            cT[j] = rb;
            if (ra < top) loc[ra - k] = where;
            if (rb < top) loc[rb - k] = j;
        }
        int cnt = 0;
        int* dst = mv + 1;
        int* src = mv + 1 + 2 * w;
        for (int t = 0; t < w; ++t)
            if (cT[t] != k + t) {
                dst[cnt] = k + t;
                src[cnt] = cT[t];
                ++cnt;
            }
        for (int s2 = 0; s2 < w; ++s2)
            if (wn[s2] >= top && cO[s2] != wn[s2]) {
                dst[cnt] = wn[s2];
                src[cnt] = cO[s2];
                ++cnt;
            }
        mv[0] = cnt;
    }
}

// One CTA per 32-column slab: read every source row segment, then write
// every destination, then overwrite the top block's panel columns with the
// factored A00 taken from the tournament root.
template <typename T>
__global__ void __launch_bounds__(256) row_move_kernel(T* __restrict__ A, int lda, int n, int k, int w,
                                                       const int* __restrict__ mv, const T* __restrict__ a00) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int cnt = mv[0];
    const int* dst = mv + 1;
    const int* src = mv + 1 + 2 * w;
    const int col = blockIdx.x * 32 + lane;
    if (col < n) {
        for (int i = warp; i < cnt; i += nwarp) tile[i * 32 + lane] = A[idx(src[i], col, lda)];
    }
    __syncthreads();
    if (col < n) {
        for (int i = warp; i < cnt; i += nwarp) A[idx(dst[i], col, lda)] = tile[i * 32 + lane];
    }
    __syncthreads();
    if (col >= k && col < k + w) {
        for (int t = warp; t < w; t += nwarp) A[idx(k + t, col, lda)] = a00[static_cast<size_t>(t) * w + (col - k)];
    }
}

template <typename T>
int pivot_apply(T* A, int lda, int m, int n, int k, int w, const int* root_list, const T* a00, int* piv, int* mv,
                cudaStream_t s) {
    (void)m;
    {
        ProfScope ps(LU_PROF_PIVOT, s);
        pivot_moves_kernel<<<1, 256, 0, s>>>(root_list, k, w, piv, mv);
        count_launches(1);
    }
    LU_LAUNCHED();
    const size_t smem = static_cast<size_t>(2 * w) * 32 * sizeof(T);
    if (int rc_ = smem_attr(row_move_kernel<T>, smem)) return rc_;
    {
        ProfScope ps(LU_PROF_PIVOT, s);
        row_move_kernel<T><<<cdiv(n, 32), 256, smem, s>>>(A, lda, n, k, w, mv, a00);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

template int pivot_apply<double>(double*, int, int, int, int, int, const int*, const double*, int*, int*,
                                 cudaStream_t);
template int pivot_apply<float>(float*, int, int, int, int, int, const int*, const float*, int*, int*, cudaStream_t);

}  // namespace lu
