// Batched LU: many independent small matrices (n <= 1024), one persistent
// launch.  Each CTA takes matrices from a queue ordered largest first and
// runs the whole blocked tournament-pivoting factorization of one matrix on
// its own (Algorithm 1 and Section 7.3 at CTA scope): leaf and playoff GEPP
// selections in shared memory, LAPACK-style row swaps, A00 from the root,
// L21 / U12 triangular solves and the Schur update.  Every update keeps the
// per-element order of the single-matrix path (fused multiply-add, pivot
// index ascending, IEEE division), so each matrix's factors equal the
// oracle's for the same panel width and leaf height.
#include "common.cuh"
#include "node_gepp.cuh"
#include "prof.cuh"
#include <climits>
#include <mutex>

namespace lu {
namespace bat {

constexpr int kThreads = 256;
constexpr int kLeaf = 128;                       // leaf height h
constexpr int kMaxN = 1024;                      // largest order taken
constexpr int kMaxB = 32;                        // largest panel width
constexpr int kMaxNodes = kMaxN / kLeaf + 1;     // first-level nodes
constexpr int kRMax = (kLeaf > 2 * kMaxB) ? kLeaf : 2 * kMaxB;   // rows a node stacks: max(h, 2b)
constexpr int kTile = 64;                        // Schur tile (64 x 64, 4 x 4 per thread)

// Panel width by size class: class c holds 2^(c+4) < n <= 2^(c+5) (class 0
// also n <= 32), c = 0..5 up to n = 1024.  The defaults are the fastest of
// 8 / 16 / 32 per class measured on GB300 (2048 matrices per class, both
// precisions): 32 everywhere, 10-17 % ahead of 16 for 129 <= n <= 512 and
// level with it (within timing noise) for n <= 64.
// lu_batched_set_panel_widths replaces them for a tuning sweep.
constexpr int kWidthClasses = 6;
struct Widths {
    int w[kWidthClasses];
};
__host__ __device__ inline int width_class(int n) {
    int c = 0;
    while (c < kWidthClasses - 1 && n > (32 << c)) ++c;
    return c;
}
__host__ __device__ inline int panel_width(const Widths& t, int n) { return t.w[width_class(n)]; }

template <typename T>
struct Smem {
    alignas(16) T W[kRMax * gepp_ws<T>(kMaxB)];  // node rows (GEPP); reused by the phases below
    T a00[kMaxB * kMaxB];                        // root's factored rows, pivot order
    int ids[kRMax];
    int ord[kRMax];
    int lists[2][kMaxNodes * kMaxB];
    int cnts[2][kMaxNodes];
    int win[kMaxB];
    int lrow[kMaxB];
    int mv[1 + 4 * kMaxB];
    GeppSlots<T> gs;
    int zero_first;
    int next;
};

// GEPP selection on the node's rows (a contiguous range or a list), panel
// columns [k, k+w).  Writes min(nr, w) row positions in pivot order to out;
// the root also leaves its factored rows in sm.a00 and records the first
// zero pivot.
template <typename T>
__device__ void node_select(Smem<T>& sm, const T* A, int lda, int k, int w, int nr, int r0, const int* list,
                            int* out, bool root) {
    const int tid = threadIdx.x;
    const int ws = gepp_ws<T>(w);
    T* W = sm.W;
    // rows in ascending position order (the blocked GEPP breaks ties by row)
    if (list) {
        for (int i = tid; i < nr; i += blockDim.x) {
            const int pi = list[i];
            int rank = 0;
            for (int j = 0; j < nr; ++j) rank += (list[j] < pi) ? 1 : 0;
            sm.ids[rank] = pi;
        }
    } else {
        for (int r = tid; r < nr; r += blockDim.x) sm.ids[r] = r0 + r;
    }
    for (int r = tid; r < nr; r += blockDim.x) sm.ord[r] = -1;
    __syncthreads();
    for (int e = tid; e < nr * w; e += blockDim.x) {
        const int r = e / w, j = e % w;
        W[r * ws + j] = A[idx(sm.ids[r], k + j, lda)];
    }
    __syncthreads();
    node_gepp_blocked<T, false, 2>(W, ws, nr, w, min(nr, w), sm.ids, sm.ord, out, sm.lrow, sm.gs,
                         root ? &sm.zero_first : nullptr);
    if (root)
        for (int e = tid; e < nr * w; e += blockDim.x) {
            const int r = e / w, j = e % w;
            const int o = sm.ord[r];
            if (o >= 0) sm.a00[o * w + j] = W[r * ws + j];
        }
    __syncthreads();
}

// TournPivot for rows [k, n), panel [k, k+w) -> sm.win (pivot order) and sm.a00.
template <typename T>
__device__ void tournament(Smem<T>& sm, const T* A, int lda, int n, int k, int w) {
    const int tid = threadIdx.x;
    const int nact = n - k;
    int H = kLeaf;
    if (kLeaf <= w) {
        H = kLeaf;
        while (H <= w) H *= 2;
    }
    const int nsuper = cdiv(nact, H);
    int cur = 0;
    for (int node = 0; node < nsuper; ++node) {
        const int r0 = k + node * H, nr = min(H, n - r0);
        int* out = &sm.lists[cur][node * w];
        if (nr > w || nsuper == 1) {
            node_select(sm, A, lda, k, w, nr, r0, nullptr, out, nsuper == 1);
            if (tid == 0) sm.cnts[cur][node] = min(nr, w);
        } else {
            for (int i = tid; i < nr; i += blockDim.x) out[i] = r0 + i;
            if (tid == 0) sm.cnts[cur][node] = nr;
        }
        __syncthreads();
    }
    int nn = nsuper;
    while (nn > 1) {
        const int npar = (nn + 1) / 2;
        for (int pnode = 0; pnode < npar; ++pnode) {
            const int l = 2 * pnode, r = 2 * pnode + 1;
            int* out = &sm.lists[cur ^ 1][pnode * w];
            const int cl = sm.cnts[cur][l];
            if (r >= nn) {
                for (int i = tid; i < cl; i += blockDim.x) out[i] = sm.lists[cur][l * w + i];
                if (tid == 0) sm.cnts[cur ^ 1][pnode] = cl;
                __syncthreads();
                continue;
            }
            const int cr = sm.cnts[cur][r];
            // the node's candidates: the left child's list, then the right child's
            __shared__ int stk[2 * kMaxB];
            for (int i = tid; i < cl; i += blockDim.x) stk[i] = sm.lists[cur][l * w + i];
            for (int i = tid; i < cr; i += blockDim.x) stk[cl + i] = sm.lists[cur][r * w + i];
            __syncthreads();
            node_select(sm, A, lda, k, w, cl + cr, 0, stk, out, npar == 1);
            if (tid == 0) sm.cnts[cur ^ 1][pnode] = min(cl + cr, w);
            __syncthreads();
        }
        cur ^= 1;
        nn = npar;
    }
    for (int i = tid; i < w; i += blockDim.x) sm.win[i] = sm.lists[cur][i];
    __syncthreads();
}

// Winners to rows k..k+w-1 by sequential swaps (one thread), then the row
// moves over all n columns, then A00 from the root.
template <typename T>
__device__ void apply_pivots(Smem<T>& sm, T* A, int lda, int n, int k, int w, int* piv) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        int cT[kMaxB], cO[kMaxB], loc[kMaxB];
        const int top = k + w;
        for (int t = 0; t < w; ++t) {
            cT[t] = k + t;
            loc[t] = t;
            cO[t] = sm.win[t];
        }
        for (int j = 0; j < w; ++j) {
            const int o = sm.win[j];
            const int where = (o >= top) ? -(j + 1) : loc[o - k];
            const int p = (where >= 0) ? (k + where) : sm.win[-where - 1];
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
        int* dst = sm.mv + 1;
        int* src = sm.mv + 1 + 2 * kMaxB;
        for (int t = 0; t < w; ++t)
            if (cT[t] != k + t) {
                dst[cnt] = k + t;
                src[cnt] = cT[t];
                ++cnt;
            }
        for (int j = 0; j < w; ++j)
            if (sm.win[j] >= top && cO[j] != sm.win[j]) {
                dst[cnt] = sm.win[j];
                src[cnt] = cO[j];
                ++cnt;
            }
        sm.mv[0] = cnt;
    }
    __syncthreads();
    const int cnt = sm.mv[0];
    const int* dst = sm.mv + 1;
    const int* src = sm.mv + 1 + 2 * kMaxB;
    T* tile = sm.W;                                      // cnt x 32
    for (int c0 = 0; c0 < n; c0 += 32) {
        for (int e = tid; e < cnt * 32; e += blockDim.x) {
            const int i = e / 32, cc = e % 32;
            if (c0 + cc < n) tile[e] = A[idx(src[i], c0 + cc, lda)];
        }
        __syncthreads();
        for (int e = tid; e < cnt * 32; e += blockDim.x) {
            const int i = e / 32, cc = e % 32;
            if (c0 + cc < n) A[idx(dst[i], c0 + cc, lda)] = tile[e];
        }
        __syncthreads();
    }
    for (int e = tid; e < w * w; e += blockDim.x) A[idx(k + e / w, k + e % w, lda)] = sm.a00[e];
    __syncthreads();
}

// L21 = A21 U00^{-1} (thread per row), U12 = L00^{-1} A12 (thread per column).
template <typename T>
__device__ void panel_solves(Smem<T>& sm, T* A, int lda, int n, int k, int w) {
    const int tid = threadIdx.x;
    T* D = sm.W;                                         // w x (w+1): the factored A00
    for (int e = tid; e < w * w; e += blockDim.x) D[(e / w) * (w + 1) + e % w] = A[idx(k + e / w, k + e % w, lda)];
    __syncthreads();
    for (int r = k + w + tid; r < n; r += blockDim.x) {
        T x[kMaxB];
#pragma unroll
        for (int j = 0; j < kMaxB; ++j) x[j] = j < w ? A[idx(r, k + j, lda)] : T(0);
#pragma unroll
        for (int j = 0; j < kMaxB; ++j) {
            if (j < w) {
                const T u = D[j * (w + 1) + j];
                x[j] = (u != T(0)) ? x[j] / u : T(0);
#pragma unroll
                for (int c = j + 1; c < kMaxB; ++c)
                    if (c < w) x[c] = fma(-x[j], D[j * (w + 1) + c], x[c]);
            }
        }
#pragma unroll
        for (int j = 0; j < kMaxB; ++j)
            if (j < w) A[idx(r, k + j, lda)] = x[j];
    }
    for (int c = k + w + tid; c < n; c += blockDim.x) {
        T x[kMaxB];
#pragma unroll
        for (int i = 0; i < kMaxB; ++i) x[i] = i < w ? A[idx(k + i, c, lda)] : T(0);
#pragma unroll
        for (int p = 0; p < kMaxB; ++p)
#pragma unroll
            for (int i = p + 1; i < kMaxB; ++i)
                if (i < w) x[i] = fma(-D[i * (w + 1) + p], x[p], x[i]);
#pragma unroll
        for (int i = 1; i < kMaxB; ++i)
            if (i < w) A[idx(k + i, c, lda)] = x[i];
    }
    __syncthreads();
}

// A22 -= L21 U12 in 64 x 64 tiles, 4 x 4 accumulators per thread, p ascending.
template <typename T>
__device__ void schur(Smem<T>& sm, T* A, int lda, int n, int k, int w) {
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = k + w, M = n - r0;
    if (M <= 0) return;
    T* Ls = sm.W;                                        // kTile x (kMaxB + 1)
    T* Us = sm.W + kTile * (kMaxB + 1);                  // kMaxB x kTile
    const int tiles = cdiv(M, kTile);
    for (int tr = 0; tr < tiles; ++tr) {
        const int i0 = r0 + tr * kTile;
        __syncthreads();
        for (int e = tid; e < kTile * w; e += blockDim.x) {
            const int i = e / w, p = e % w;
            Ls[i * (kMaxB + 1) + p] = (i0 + i < n) ? A[idx(i0 + i, k + p, lda)] : T(0);
        }
        for (int tc = 0; tc < tiles; ++tc) {
            const int j0 = r0 + tc * kTile;
            // the tile's current values first: their loads fly while U12's
            // columns are staged
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
                    acc[a][b] = (i < n && j < n) ? A[idx(i, j, lda)] : T(0);
                }
            __syncthreads();
            for (int e = tid; e < w * kTile; e += blockDim.x) {
                const int p = e / kTile, j = e % kTile;
                Us[p * kTile + j] = (j0 + j < n) ? A[idx(k + p, j0 + j, lda)] : T(0);
            }
            __syncthreads();
            for (int p = 0; p < w; ++p) {
                T lv[4], uv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) lv[a] = Ls[(ty + 16 * a) * (kMaxB + 1) + p];
#pragma unroll
                for (int b = 0; b < 4; ++b) uv[b] = Us[p * kTile + tx + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(-lv[a], uv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
                    if (i < n && j < n) A[idx(i, j, lda)] = acc[a][b];
                }
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) batched_lu_kernel(int batch, const int* __restrict__ ns,
                                                              T* const* __restrict__ As, const int* __restrict__ ldas,
                                                              int* const* __restrict__ pivs, int* __restrict__ info,
                                                              const int* __restrict__ order, int* __restrict__ counter,
                                                              Widths widths) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) sm.next = atomicAdd(counter, 1);
        __syncthreads();
        const int t = sm.next;
        __syncthreads();
        if (t >= batch) break;
        const int mi = order[t];
        const int n = ns[mi];
        T* A = As[mi];
        const int lda = ldas[mi];
        int* piv = pivs[mi];
        if (n < 0 || n > kMaxN || (n > 0 && (A == nullptr || piv == nullptr || lda < n))) {
            if (threadIdx.x == 0) info[mi] = -1;
            continue;
        }
        if (threadIdx.x == 0) sm.zero_first = -1;
        int first_zero = -1;
        const int b = panel_width(widths, n);
        for (int k = 0; k < n; k += b) {
            const int w = min(b, n - k);
            tournament(sm, A, lda, n, k, w);
            if (threadIdx.x == 0 && first_zero < 0 && sm.zero_first >= 0) first_zero = k + sm.zero_first;
            if (threadIdx.x == 0) sm.zero_first = -1;
            apply_pivots(sm, A, lda, n, k, w, piv);
            panel_solves(sm, A, lda, n, k, w);
            schur(sm, A, lda, n, k, w);
        }
        if (threadIdx.x == 0) info[mi] = first_zero >= 0 ? first_zero + 1 : 0;
        __syncthreads();
    }
}

// Largest-first order by a counting sort on n (sizes outside [0, kMaxN] go last).
__global__ void size_hist_kernel(int batch, const int* __restrict__ ns, int* __restrict__ hist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        const int n = ns[i];
        const int key = (n >= 0 && n <= kMaxN) ? kMaxN - n : kMaxN + 1;
        atomicAdd(&hist[key], 1);
    }
}
__global__ void size_scan_kernel(int* __restrict__ hist, int* __restrict__ counter) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i <= kMaxN + 1; ++i) {
            const int c = hist[i];
            hist[i] = s;
            s += c;
        }
        *counter = 0;
    }
}
__global__ void size_scatter_kernel(int batch, const int* __restrict__ ns, int* __restrict__ hist,
                                    int* __restrict__ order) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        const int n = ns[i];
        const int key = (n >= 0 && n <= kMaxN) ? kMaxN - n : kMaxN + 1;
        order[atomicAdd(&hist[key], 1)] = i;
    }
}

// ---------------------------------------------------------------------------
// Batched solve: X = U^{-1} L^{-1} P B per matrix, one CTA per matrix, one
// warp per right-hand side (row dot products across the lanes).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) batched_solve_kernel(int batch, const int* __restrict__ ns,
                                                                 const int* __restrict__ nrhss,
                                                                 T* const* __restrict__ LUs, const int* __restrict__ ldas,
                                                                 int* const* __restrict__ pivs, T* const* __restrict__ Bs,
                                                                 const int* __restrict__ ldbs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ybuf = reinterpret_cast<T*>(smem_raw);            // 8 x kMaxN
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int mi = blockIdx.x; mi < batch; mi += gridDim.x) {
        const int n = ns[mi], nr = nrhss[mi];
        if (n <= 0 || n > kMaxN || nr <= 0 || nr > 8) continue;
        const T* LU = LUs[mi];
        const int lda = ldas[mi];
        const int* piv = pivs[mi];
        T* B = Bs[mi];
        const int ldb = ldbs[mi];
        if (warp < nr) {
            T* yc = ybuf + static_cast<size_t>(warp) * kMaxN;
            for (int i = lane; i < n; i += 32) yc[i] = B[idx(i, warp, ldb)];
            __syncwarp();
            if (lane == 0)
                for (int i = 0; i < n; ++i) {
                    const int p = piv[i];
                    const T t = yc[i];
                    yc[i] = yc[p];
                    yc[p] = t;
                }
            __syncwarp();
            for (int i = 1; i < n; ++i) {                // forward, unit L
                T s = 0;
                for (int p = lane; p < i; p += 32) s = fma(LU[idx(i, p, lda)], yc[p], s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) yc[i] -= s;
                __syncwarp();
            }
            for (int i = n - 1; i >= 0; --i) {           // backward, U
                T s = 0;
                for (int p = i + 1 + lane; p < n; p += 32) s = fma(LU[idx(i, p, lda)], yc[p], s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) yc[i] = (yc[i] - s) / LU[idx(i, i, lda)];
                __syncwarp();
            }
            for (int i = lane; i < n; i += 32) B[idx(i, warp, ldb)] = yc[i];
        }
        __syncthreads();
    }
}

// measured defaults per dtype (index 0 binary64, 1 binary32) and the
// table in use
constexpr Widths kDefaultWidths[2] = {{{32, 32, 32, 32, 32, 32}}, {{32, 32, 32, 32, 32, 32}}};
static std::mutex g_width_mu;
static Widths g_widths[2] = {kDefaultWidths[0], kDefaultWidths[1]};

static Widths widths_for(int dtype) {
    std::lock_guard<std::mutex> lk(g_width_mu);
    return g_widths[dtype == LU_PREC_F32 ? 1 : 0];
}

}  // namespace bat

static int sms() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

template <typename T>
static int factor_batched(int batch, const int* n, T* const* A, const int* lda, int* const* piv, int* info,
                          const bat::Widths& widths, cudaStream_t s) {
    int* ws = nullptr;
    const size_t words = static_cast<size_t>(batch) + (bat::kMaxN + 2) + 4;
    if (lu_malloc_async(reinterpret_cast<void**>(&ws), words * sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    int* order = ws;
    int* hist = ws + batch;
    int* counter = hist + bat::kMaxN + 2;
    int rc = 0;
    if (cudaMemsetAsync(hist, 0, (bat::kMaxN + 2) * sizeof(int), s) != cudaSuccess) rc = LU_ELAUNCH;
    if (!rc) {
        ProfScope ps(LU_PROF_OTHER, s);
        bat::size_hist_kernel<<<cdiv(batch, 256), 256, 0, s>>>(batch, n, hist);
        bat::size_scan_kernel<<<1, 32, 0, s>>>(hist, counter);
        bat::size_scatter_kernel<<<cdiv(batch, 256), 256, 0, s>>>(batch, n, hist, order);
        count_launches(3);
        if (cudaPeekAtLastError() != cudaSuccess) rc = LU_ELAUNCH;
    }
    if (!rc) {
        const size_t smem = sizeof(bat::Smem<T>);
        rc = smem_attr(bat::batched_lu_kernel<T>, smem);
        int per_sm = 0;
        if (!rc && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bat::batched_lu_kernel<T>, bat::kThreads,
                                                                 smem) != cudaSuccess)
            rc = LU_ELAUNCH;
        if (!rc) {
            const int grid = sms() * (per_sm > 0 ? per_sm : 1);
            ProfScope ps(LU_PROF_SCHUR, s);
            bat::batched_lu_kernel<T><<<grid < batch ? grid : batch, bat::kThreads, smem, s>>>(batch, n, A, lda, piv,
                                                                                              info, order, counter,
                                                                                              widths);
            count_launches(1);
            if (cudaPeekAtLastError() != cudaSuccess) rc = LU_ELAUNCH;
        }
    }
    cudaGetLastError();
    cudaFreeAsync(ws, s);
    return rc;
}

}  // namespace lu

using namespace lu;

extern "C" int lu_batched_panel_width(int n) { return bat::panel_width(bat::widths_for(LU_PREC_F64), n); }

extern "C" int lu_batched_panel_width_dt(int n, int dtype) {
    if (dtype != LU_PREC_F64 && dtype != LU_PREC_F32) return -2;
    return bat::panel_width(bat::widths_for(dtype), n);
}

extern "C" int lu_batched_set_panel_widths(int dtype, const int* widths, int count) {
    if (dtype != LU_PREC_F64 && dtype != LU_PREC_F32) return -1;
    const int d = dtype == LU_PREC_F32 ? 1 : 0;
    if (widths == nullptr) {
        std::lock_guard<std::mutex> lk(bat::g_width_mu);
        bat::g_widths[d] = bat::kDefaultWidths[d];
        return 0;
    }
    if (count != bat::kWidthClasses) return -3;
    bat::Widths t{};
    for (int c = 0; c < count; ++c) {
        if (widths[c] < 1 || widths[c] > bat::kMaxB) return -2;
        t.w[c] = widths[c];
    }
    std::lock_guard<std::mutex> lk(bat::g_width_mu);
    bat::g_widths[d] = t;
    return 0;
}

extern "C" int lu_factor_batched(int batch, const int* n, void* const* A, const int* lda, int* const* piv, int* info,
                                 int dtype, cudaStream_t stream) {
    if (batch < 0) return -1;
    if (batch == 0) return 0;
    if (n == nullptr) return -2;
    if (A == nullptr) return -3;
    if (lda == nullptr) return -4;
    if (piv == nullptr) return -5;
    if (info == nullptr) return -6;
    if (dtype == LU_PREC_F64)
        return factor_batched<double>(batch, n, reinterpret_cast<double* const*>(A), lda, piv, info,
                                      bat::widths_for(dtype), stream);
    if (dtype == LU_PREC_F32)
        return factor_batched<float>(batch, n, reinterpret_cast<float* const*>(A), lda, piv, info,
                                     bat::widths_for(dtype), stream);
    return -7;
}

extern "C" int lu_solve_batched(int batch, const int* n, const int* nrhs, void* const* LU, const int* lda,
                                int* const* piv, void* const* B, const int* ldb, int dtype, cudaStream_t stream) {
    if (batch < 0) return -1;
    if (batch == 0) return 0;
    if (!n || !nrhs || !LU || !lda || !piv || !B || !ldb) return -2;
    const int grid = batch < 4 * sms() ? batch : 4 * sms();
    ProfScope ps(LU_PROF_SOLVE, stream);
    if (dtype == LU_PREC_F64) {
        const size_t smem = 8 * static_cast<size_t>(bat::kMaxN) * sizeof(double);
        if (int rc_ = smem_attr(bat::batched_solve_kernel<double>, smem)) return rc_;
        bat::batched_solve_kernel<double><<<grid, bat::kThreads, smem, stream>>>(
            batch, n, nrhs, reinterpret_cast<double* const*>(LU), lda, piv, reinterpret_cast<double* const*>(B), ldb);
    } else if (dtype == LU_PREC_F32) {
        const size_t smem = 8 * static_cast<size_t>(bat::kMaxN) * sizeof(float);
        if (int rc_ = smem_attr(bat::batched_solve_kernel<float>, smem)) return rc_;
        bat::batched_solve_kernel<float><<<grid, bat::kThreads, smem, stream>>>(
            batch, n, nrhs, reinterpret_cast<float* const*>(LU), lda, piv, reinterpret_cast<float* const*>(B), ldb);
    } else {
        return -9;
    }
    count_launches(1);
    LU_LAUNCHED();
    return 0;
}
