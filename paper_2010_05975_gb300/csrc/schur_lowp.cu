// FactorizeA11 (Section 7.2) with low-precision operands on the 5th-generation
// tensor cores:  C -= sL * sU * (Lq . Uq)  where C is the binary32 trailing
// matrix, Lq / Uq are L21 / U12 rounded to bfloat16 or fp8 e4m3, and sL / sU
// are power-of-two scales, one per 256 x 256 operand tile (fp8 only; bf16
// keeps binary32's exponent range and uses scale 1).  Accumulation is fp32
// in tensor memory.  The paper is silent on precision; this is the
// mixed-precision variant of the update that the refinement solver uses.
//
// Pieces:
//   quantize_l21_kernel  L21 (rows r0.., K = w <= 256) -> Lq [M x 256], K-major
//   quantize_u12_kernel  U12 (K x columns)               -> UqT [N x 256], K-major
//   schur_tc_kernel      persistent tcgen05 GEMM, 128 x 128 tiles, K = 256
// The GEMM's warps: warp 0 issues TMA loads, warp 1 owns tensor memory and
// issues the MMAs (one elected thread), warps 2-5 run the epilogue
// (tcgen05.ld -> fused C update in global memory; each thread loads its
// row of the C tile before waiting for the accumulator).  Every mbarrier wait
// has a wall-clock deadline; a wait that runs out sets an abort flag, the CTA
// waits for its own copies and MMAs in flight, frees its tensor memory and
// exits, and the host sees info / status = -LU_ETIMEOUT.
#include "common.cuh"
#include "prof.cuh"
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <algorithm>
#include <cstring>

namespace lu {

constexpr int kTcBM = 128;        // rows of a C tile (MMA M)
constexpr int kTcBN = 128;        // columns of a C tile (MMA N)
constexpr int kTcK = 256;         // padded K of every step (b <= 256)
constexpr int kTcThreads = 192;   // 6 warps
constexpr int kScaleTile = 256;   // operand rows/columns sharing one scale
constexpr int kTsluReserveSMs = 16;           // SMs left to the concurrent tournament
constexpr int kTcStages = 3;      // operand stages (one 128-byte K chunk of A and of B each)

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait for the phase with the given parity, at most limit_ns of wall-clock
// time (%globaltimer, checked every 64 polls).  Returns false when the
// deadline passes (and raises the abort flag) or, with check_abort, when
// another role already aborted.  With check_abort false the wait ignores the
// flag: it drains copies and MMAs this CTA issued, which complete by
// themselves, before the CTA exits.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns, bool check_abort = true) {
    const uint32_t a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (uint32_t it = 1;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 0) {
            if (check_abort && *abort_flag) return false;
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
template <bool kFp8>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (kFp8) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05 format): K-major operand whose
// rows are 128 bytes, written by TMA with the 128-byte swizzle; 8-row groups
// 1024 bytes apart.  Bits: start>>4 [0,14), LBO>>4 [16,30), SBO>>4 [32,46),
// version 1 [46,48), layout 2 = SWIZZLE_128B [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
    d |= static_cast<uint64_t>(1) << 16;                   // LBO (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;           // SBO: 8 rows x 128 B
    d |= static_cast<uint64_t>(1) << 46;                   // descriptor version
    d |= static_cast<uint64_t>(2) << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: D fp32, A/B bf16 (kind::f16) or e4m3 (kind::f8f6f4),
// both K-major, M = 128, N = 128.
template <bool kFp8>
__host__ __device__ constexpr uint32_t make_idesc() {
    return (1u << 4)                                    // D format: f32
           | ((kFp8 ? 0u : 1u) << 7)                    // A: e4m3 = 0 / bf16 = 1
           | ((kFp8 ? 0u : 1u) << 10)                   // B
           | (static_cast<uint32_t>(kTcBN >> 3) << 17)  // N >> 3
           | (static_cast<uint32_t>(kTcBM >> 4) << 24); // M >> 4
}

// One pending panel of a launch, as seen from the launch's C region.
struct TcPanel {
    int rowL;            // Lq row that the region's row 0 maps to
    int rowU;            // UqT row that the region's column 0 maps to
    int nchunk;          // 128-byte K chunks holding the panel's w columns
    const int* eLrow;    // fp8: scale exponent of each Lq row (nullptr: scale 1)
    const int* eU;       // fp8: scale exponent of each 256-row block of UqT
};

// Tensor maps of a launch: C (TMA epilogue only), then Lq / UqT of each panel.
struct TcMaps {
    CUtensorMap c;
    CUtensorMap op[2 * kTcMaxPanels];
};

struct TcArgs {
    float* C;          // top-left of the region
    int ldc;
    int M, N;          // region extent
    int np;            // pending panels applied, in this order (1..kTcMaxPanels)
    TcPanel p[kTcMaxPanels];
    int* status;       // set to -LU_ETIMEOUT on a timed-out wait
    int tma_c;         // C moves through TMA (16-byte aligned rows) or per-thread loads
    unsigned long long wait_ns;   // deadline of one dependency wait
    int inject;        // test hook: the MMA warp first waits on a barrier nothing arrives on
};

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// C -= sum_p s_p (Lq_p . Uq_p^T) over the region, one 128 x 128 C tile at a
// time, each pending panel p into its own tensor-memory accumulator; the
// epilogue applies the panels in order, C = fma(-s_p, acc_p, C), so every
// element gets the same rounding sequence as one launch per panel.
template <bool kFp8>
__global__ void __launch_bounds__(kTcThreads, 1) schur_tc_kernel(const __grid_constant__ TcMaps maps, TcArgs a) {
    constexpr int kElem = kFp8 ? 1 : 2;
    constexpr int kKBlk = 128 / kElem;                     // K elements per 128-byte chunk
    constexpr int kMmaK = 32 / kElem;                      // K per MMA instruction (32 bytes)
    constexpr uint32_t kChunkBytes = 128 * 128;            // 128 rows x 128 bytes
    constexpr uint32_t kStageBytes = 2 * kChunkBytes;      // A chunk + B chunk
    constexpr uint32_t kCBufBytes = kTcBM * kTcBN * 4;     // one C tile (4 boxes of 32 columns)
    constexpr uint32_t kIdesc = make_idesc<kFp8>();

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sC = base;                                  // [2] C tiles (TMA epilogue)
    unsigned char* sOp = base + 2 * kCBufBytes;                // [kTcStages] operand stages
    uint64_t* bars = reinterpret_cast<uint64_t*>(sOp + kTcStages * kStageBytes);
    uint64_t* full = bars;                                     // [kTcStages]
    uint64_t* empty = bars + kTcStages;                        // [kTcStages]
    uint64_t* acc_full = bars + 2 * kTcStages;                 // [2]
    uint64_t* acc_empty = acc_full + 2;                        // [2]
    uint64_t* c_full = acc_empty + 2;                          // [2]
    uint64_t* mma_done = c_full + 2;
    uint64_t* never = mma_done + 1;                            // test hook: no thread ever arrives here
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
    __shared__ int s_abort;
    __shared__ int s_go;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = a.np;
    const int nbuf = np <= 2 ? 2 : 1;                          // accumulator sets in flight
    const uint32_t ncols = (nbuf * np * kTcBN <= 256) ? 256u : 512u;
    const int MB = cdiv(a.M, kTcBM), NB = cdiv(a.N, kTcBN);
    const long long T = static_cast<long long>(MB) * NB;
    const long long t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(acc_full + i, 1);
            mbar_init(acc_empty + i, 128);
            mbar_init(c_full + i, 1);
        }
        mbar_init(mma_done, 1);
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---------------- operand producer: (tile, panel, K chunk) ----------------
        long long q = 0;
        bool ok = true;
        for (long long t = t0; ok && t < t1; ++t) {
            const int mb = static_cast<int>(t / NB), nb = static_cast<int>(t % NB);
            for (int pi = 0; ok && pi < np; ++pi) {
                const TcPanel& P = a.p[pi];
                for (int kc = 0; kc < P.nchunk; ++kc, ++q) {
                    const int st = static_cast<int>(q % kTcStages);
                    const long long round = q / kTcStages;
                    if (round > 0 && !mbar_wait(empty + st, static_cast<uint32_t>((round - 1) & 1), abort_flag, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    unsigned char* sA = sOp + st * kStageBytes;
                    mbar_expect_tx(full + st, kStageBytes);
                    tma_load_2d(sA, &maps.op[2 * pi], kc * kKBlk, P.rowL + mb * kTcBM, full + st);
                    tma_load_2d(sA + kChunkBytes, &maps.op[2 * pi + 1], kc * kKBlk, P.rowU + nb * kTcBN, full + st);
                }
            }
        }
        // No CTA exit with TMA writes in flight: wait for the last load of
        // every stage (complete already unless another role aborted before
        // consuming it).
        for (int st = 0; st < kTcStages; ++st) {
            const long long uses = q > st ? (q - 1 - st) / kTcStages + 1 : 0;
            if (uses > 0) mbar_wait(full + st, static_cast<uint32_t>((uses - 1) & 1), abort_flag, kDrainWaitNs, false);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        long long q = 0;
        bool ok = !a.inject || mbar_wait(never, 0, abort_flag, a.wait_ns);
        for (long long t = t0; ok && t < t1; ++t) {
            const int it = static_cast<int>(t - t0);
            const int buf = nbuf == 2 ? (it & 1) : 0;
            const int use = nbuf == 2 ? (it >> 1) : it;
            if (use > 0 && !mbar_wait(acc_empty + buf, static_cast<uint32_t>((use - 1) & 1), abort_flag, a.wait_ns)) break;
            tc_fence_after();
            for (int pi = 0; ok && pi < np; ++pi) {
                const uint32_t d = tmem + static_cast<uint32_t>((buf * np + pi) * kTcBN);
                for (int kc = 0; kc < a.p[pi].nchunk; ++kc, ++q) {
                    const int st = static_cast<int>(q % kTcStages);
                    if (!mbar_wait(full + st, static_cast<uint32_t>((q / kTcStages) & 1), abort_flag, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aB = smem_u32(sOp + st * kStageBytes), bB = aB + kChunkBytes;
#pragma unroll
                    for (int kk = 0; kk < kKBlk / kMmaK; ++kk)
                        tc_mma<kFp8>(d, sw128_desc(aB + kk * 32), sw128_desc(bB + kk * 32), kIdesc,
                                     (kc | kk) ? 1u : 0u);
                    tc_commit(empty + st);
                }
            }
            if (ok) tc_commit(acc_full + buf);
        }
        // every MMA issued so far has completed once mma_done flips
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, abort_flag, kDrainWaitNs, false);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int qd = warp & 3;                 // TMEM lane quarter this warp may access
        const int rl = qd * 32 + lane;           // row of the tile this thread owns
        const bool leader = (warp == 2 && lane == 0);
        if (a.tma_c) {
            // C tiles through shared memory: TMA load -> per-row update ->
            // TMA store.  The leader issues the copies and makes the waits;
            // a named barrier hands its verdict to all 128 threads, so they
            // leave the loop together.
            // boxes of 32 columns that start inside the region (a copy never
            // starts past the last column)
            auto nbox = [&](long long t) { return min(4, cdiv(a.N - static_cast<int>(t % NB) * kTcBN, 32)); };
            auto load_c = [&](long long t, int b2) {
                const int nbx = nbox(t);
                mbar_expect_tx(c_full + b2, static_cast<uint32_t>(nbx) * (kCBufBytes / 4));
                for (int j = 0; j < nbx; ++j)
                    tma_load_2d(sC + b2 * kCBufBytes + j * (kCBufBytes / 4), &maps.c,
                                static_cast<int>(t % NB) * kTcBN + 32 * j, static_cast<int>(t / NB) * kTcBM,
                                c_full + b2);
            };
            int loads = 0;
            if (leader && t0 < t1) {
                load_c(t0, 0);
                loads = 1;
            }
            for (long long t = t0; t < t1; ++t) {
                const int it = static_cast<int>(t - t0);
                const int cb = it & 1;
                const int buf = nbuf == 2 ? (it & 1) : 0;
                const int use = nbuf == 2 ? (it >> 1) : it;
                const int mb = static_cast<int>(t / NB), nb = static_cast<int>(t % NB);
                if (leader) {
                    bool ok = true;
                    if (t + 1 < t1) {
                        // the other buffer's last store (tile it - 1) has been read out
                        bulk_wait_read_all();
                        load_c(t + 1, cb ^ 1);
                        ++loads;
                    }
                    ok = mbar_wait(c_full + cb, static_cast<uint32_t>((it >> 1) & 1), abort_flag, a.wait_ns) &&
                         mbar_wait(acc_full + buf, static_cast<uint32_t>(use & 1), abort_flag, a.wait_ns);
                    s_go = ok ? 1 : 0;
                }
                epi_sync();
                if (!s_go) break;
                tc_fence_after();
                const int r = mb * kTcBM + rl;
                float sc[kTcMaxPanels];
#pragma unroll
                for (int pi = 0; pi < kTcMaxPanels; ++pi) {
                    int e = 0;
                    if (pi < np) {
                        if (a.p[pi].eLrow && r < a.M) e += a.p[pi].eLrow[a.p[pi].rowL + r];
                        if (a.p[pi].eU) e += a.p[pi].eU[(a.p[pi].rowU + nb * kTcBN) / kScaleTile];
                    }
                    sc[pi] = ldexpf(1.0f, e);
                }
                unsigned char* ctile = sC + cb * kCBufBytes;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // row rl of box j: 8 16-byte chunks, 128-byte swizzle
                    float4* row = reinterpret_cast<float4*>(ctile + j * (kCBufBytes / 4) + rl * 128);
                    float4 x[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) x[c] = row[c ^ (rl & 7)];
#pragma unroll
                    for (int pi = 0; pi < kTcMaxPanels; ++pi) {
                        if (pi < np) {
                            float v[32];
                            tmem_ld32(tmem + (static_cast<uint32_t>(qd * 32) << 16) +
                                          static_cast<uint32_t>((buf * np + pi) * kTcBN + 32 * j),
                                      v);
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                x[c].x = fmaf(-sc[pi], v[4 * c + 0], x[c].x);
                                x[c].y = fmaf(-sc[pi], v[4 * c + 1], x[c].y);
                                x[c].z = fmaf(-sc[pi], v[4 * c + 2], x[c].z);
                                x[c].w = fmaf(-sc[pi], v[4 * c + 3], x[c].w);
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) row[c ^ (rl & 7)] = x[c];
                }
                tc_fence_before();
                mbar_arrive(acc_empty + buf);
                proxy_fence_smem();
                epi_sync();
                if (leader) {
                    const int nbx = nbox(t);
                    for (int j = 0; j < nbx; ++j)
                        tma_store_2d(&maps.c, nb * kTcBN + 32 * j, mb * kTcBM, ctile + j * (kCBufBytes / 4));
                    bulk_commit();
                }
            }
            if (leader) {
                // every C load issued has landed (an abort can leave the
                // prefetch unconsumed) and every store has completed
                for (int b2 = 0; b2 < 2; ++b2) {
                    const int nl = loads > b2 ? (loads - 1 - b2) / 2 + 1 : 0;
                    if (nl > 0) mbar_wait(c_full + b2, static_cast<uint32_t>((nl - 1) & 1), abort_flag, kDrainWaitNs, false);
                }
                bulk_wait_all();
            }
        } else {
            // C rows not 16-byte aligned: each thread reads and writes its own
            // row, 32 columns at a time.
            for (long long t = t0; t < t1; ++t) {
                const int it = static_cast<int>(t - t0);
                const int buf = nbuf == 2 ? (it & 1) : 0;
                const int use = nbuf == 2 ? (it >> 1) : it;
                const int mb = static_cast<int>(t / NB), nb = static_cast<int>(t % NB);
                const int r = mb * kTcBM + rl;
                if (!mbar_wait(acc_full + buf, static_cast<uint32_t>(use & 1), abort_flag, a.wait_ns)) break;
                tc_fence_after();
                float* crow = a.C + idx(r < a.M ? r : 0, nb * kTcBN, a.ldc);
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    const int cmax = a.N - nb * kTcBN - 32 * j;       // valid columns in this chunk
                    float x[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) x[i] = (r < a.M && i < cmax) ? crow[32 * j + i] : 0.0f;
                    for (int pi = 0; pi < np; ++pi) {
                        float v[32];
                        tmem_ld32(tmem + (static_cast<uint32_t>(qd * 32) << 16) +
                                      static_cast<uint32_t>((buf * np + pi) * kTcBN + 32 * j),
                                  v);
                        int e = a.p[pi].eU ? a.p[pi].eU[(a.p[pi].rowU + nb * kTcBN) / kScaleTile] : 0;
                        if (a.p[pi].eLrow && r < a.M) e += a.p[pi].eLrow[a.p[pi].rowL + r];
                        const float sc = ldexpf(1.0f, e);
#pragma unroll
                        for (int i = 0; i < 32; ++i) x[i] = fmaf(-sc, v[i], x[i]);
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (r < a.M && i < cmax) crow[32 * j + i] = x[i];
                }
                tc_fence_before();
                mbar_arrive(acc_empty + buf);
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
    if (threadIdx.x == 0 && s_abort) atomicExch(a.status, -LU_ETIMEOUT);
}

// ----------------------------------------------------------------------------
// Quantization
// ----------------------------------------------------------------------------
template <bool kFp8>
__device__ __forceinline__ void store_q(unsigned char* dst, size_t i, float x) {
    if constexpr (kFp8) {
        dst[i] = static_cast<unsigned char>(__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3));
    } else {
        reinterpret_cast<__nv_bfloat16*>(dst)[i] = __float2bfloat16_rn(x);
    }
}

// Power-of-two exponent e with maxabs * 2^-e <= 448 (e4m3's largest finite).
__device__ __forceinline__ int fp8_exponent(float maxabs) {
    if (!(maxabs > 0.0f) || !(maxabs < INFINITY)) return 0;
    int ex;
    const float f = frexpf(maxabs / 448.0f, &ex);
    return (f == 0.5f) ? ex - 1 : ex;
}

__device__ __forceinline__ float block_max(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (blockDim.x >> 5) ? red[lane] : 0.0f;
        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
}

// Eight binary32 values from p (16-byte aligned when vec), zero at and past
// column limit `lim` of the row.
__device__ __forceinline__ void load8(const float* p, int c, int lim, bool vec, float (&v)[8]) {
    if (vec && c + 8 <= lim) {
        const float4 a = *reinterpret_cast<const float4*>(p + c), b = *reinterpret_cast<const float4*>(p + c + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (c + i < lim) ? p[c + i] : 0.0f;
    }
}

// 8 values -> 8 bf16 (16 bytes) or 8 e4m3 (8 bytes) at dst (aligned)
template <bool kFp8>
__device__ __forceinline__ void store8(unsigned char* dst, const float (&v)[8], int e) {
    if constexpr (kFp8) {
        uint32_t w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            w[h] = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                w[h] |= static_cast<uint32_t>(__nv_cvt_float_to_fp8(ldexpf(v[4 * h + i], -e), __NV_SATFINITE, __NV_E4M3))
                        << (8 * i);
        }
        *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    } else {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i]));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i + 1]));
            w[i] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// L21 = A[r0 .. r0+M, k .. k+w) -> Lq [M x 256] (K-major), columns [w, kpad)
// zero (kpad = w rounded up to a 128-byte chunk), later columns never read.
// fp8: one power-of-two scale per 256-row block, counted from r0; every row
// records its block's exponent (eLrow), so that the row can later move (a
// pivot swap of a deferred panel) and keep the scale it was rounded with.
// One CTA per 256-row block (fp8) or 64 rows (bf16); 8 consecutive K-values
// per thread and step.
template <bool kFp8>
__global__ void __launch_bounds__(512) quantize_l21_kernel(const float* __restrict__ A, int lda, int r0, int M, int k,
                                                           int w, int kpad, int vec, unsigned char* __restrict__ Lq,
                                                           int* __restrict__ eLrow) {
    __shared__ float red[32];
    constexpr int kElem = kFp8 ? 1 : 2;
    constexpr int kRB = kFp8 ? kScaleTile : 64;     // rows per CTA (a whole scale block for fp8)
    const int rb = blockIdx.x * kRB;
    const int nr = min(kRB, M - rb);
    const int tpr = kpad / 8;                       // threads per row
    const int rpp = blockDim.x / tpr;               // rows per pass
    const int tr = threadIdx.x / tpr, c = (threadIdx.x % tpr) * 8;
    int e = 0;
    if constexpr (kFp8) {
        float mx = 0.0f;
        for (int i = tr; i < nr; i += rpp) {
            float v[8];
            load8(A + idx(r0 + rb + i, k, lda), c, w, vec != 0, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) mx = fmaxf(mx, fabsf(v[q]));
        }
        mx = block_max(mx, red);
        e = fp8_exponent(mx);
        for (int i = threadIdx.x; i < nr; i += blockDim.x) eLrow[rb + i] = e;
    }
    for (int i = tr; i < nr; i += rpp) {
        float v[8];
        load8(A + idx(r0 + rb + i, k, lda), c, w, vec != 0, v);
        store8<kFp8>(Lq + (static_cast<size_t>(rb + i) * kTcK + c) * kElem, v, e);
    }
}

// U12 = A[k .. k+w, c0 .. c0+N) -> UqT [N x 256] (transposed: K-major),
// columns [w, kpad) zero.  fp8: one scale per 256 columns.  One CTA per 256
// columns (fp8) or per 64 (bf16); 64-column chunks are staged transposed in
// shared memory, then written 8 K-values per thread.
template <bool kFp8>
__global__ void __launch_bounds__(512) quantize_u12_kernel(const float* __restrict__ A, int lda, int k, int w, int c0,
                                                           int N, int kpad, int vec, unsigned char* __restrict__ Uq,
                                                           int* __restrict__ expU) {
    __shared__ float red[32];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tile = reinterpret_cast<float*>(smem_raw);            // [64][kpad + 1]: tile[col][kk]
    constexpr int kElem = kFp8 ? 1 : 2;
    constexpr int kCols = kFp8 ? kScaleTile : 64;                // columns per CTA
    const int cb = blockIdx.x * kCols;
    const int nc = min(kCols, N - cb);
    const int ts = kpad + 1;
    int e = 0;
    if constexpr (kFp8) {
        float mx = 0.0f;
        // rows kk < w, 8 columns per thread
        const int tpr = kCols / 8;
        for (int i = threadIdx.x; i < w * tpr; i += blockDim.x) {
            const int kk = i / tpr, cc = (i % tpr) * 8;
            float v[8];
            load8(A + idx(k + kk, c0 + cb, lda), cc, nc, vec != 0, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) mx = fmaxf(mx, fabsf(v[q]));
        }
        mx = block_max(mx, red);
        e = fp8_exponent(mx);
        if (threadIdx.x == 0) expU[blockIdx.x] = e;
    }
    for (int ch = 0; ch < nc; ch += 64) {
        const int ncc = min(64, nc - ch);
        // rows kk < kpad of the 64-column chunk, transposed (zero past w)
        for (int i = threadIdx.x; i < kpad * 8; i += blockDim.x) {
            const int kk = i / 8, cc = (i % 8) * 8;
            float v[8];
            if (kk < w) {
                load8(A + idx(k + kk, c0 + cb + ch, lda), cc, ncc, vec != 0, v);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) tile[(cc + q) * ts + kk] = v[q];
        }
        __syncthreads();
        const int tpc = kpad / 8;                               // threads per column
        for (int i = threadIdx.x; i < ncc * tpc; i += blockDim.x) {
            const int col = i / tpc, kk = (i % tpc) * 8;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = tile[col * ts + kk + q];
            store8<kFp8>(Uq + (static_cast<size_t>(cb + ch + col) * kTcK + kk) * kElem, v, e);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// rows x 256 K-major operand, box = 128 rows x 128 bytes, 128-byte swizzle.
static int make_operand_map(CUtensorMap* map, const void* base, int rows, bool fp8) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return LU_ELAUNCH;
    const int elem = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kTcK), static_cast<cuuint64_t>(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kTcK) * elem};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem), 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : LU_ELAUNCH;
}

// The C region (M x N binary32, row stride ldc) as boxes of 128 rows x 32
// columns (128 bytes), 128-byte swizzle.  Out-of-range rows and columns read
// as zero and are not written back.
static int make_c_map(CUtensorMap* map, float* C, int ldc, int M, int N) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return LU_ELAUNCH;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(M)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldc) * sizeof(float)};
    cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTcBM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : LU_ELAUNCH;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

size_t lowp_smem_bytes() {
    return 1024 + 2 * static_cast<size_t>(kTcBM) * kTcBN * 4 + static_cast<size_t>(kTcStages) * 2 * 128 * 128 + 256;
}

int lowp_kpad(int w, bool fp8) {
    const int kb = fp8 ? 128 : 64;
    return (w + kb - 1) / kb * kb;
}

int quantize_l21(const float* A, int lda, int m, int k, int w, bool fp8, void* Lq, int* eLrow, cudaStream_t s) {
    const int r0 = k + w, M = m - r0;
    if (M <= 0) return 0;
    const int kpad = lowp_kpad(w, fp8);
    const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 3) == 0 && (k & 3) == 0) ? 1 : 0;
    {
        ProfScope ps(LU_PROF_OTHER, s);
        if (fp8)
            quantize_l21_kernel<true><<<cdiv(M, kScaleTile), 512, 0, s>>>(A, lda, r0, M, k, w, kpad, vec,
                                                                           static_cast<unsigned char*>(Lq), eLrow);
        else
            quantize_l21_kernel<false><<<cdiv(M, 64), 512, 0, s>>>(A, lda, r0, M, k, w, kpad, vec,
                                                                            static_cast<unsigned char*>(Lq), eLrow);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

int quantize_u12(const float* A, int lda, int k, int w, int c0, int c1, bool fp8, void* Uq, int* expU,
                 cudaStream_t s) {
    const int N = c1 - c0;
    if (N <= 0) return 0;
    const int kpad = lowp_kpad(w, fp8);
    const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 3) == 0 && (c0 & 3) == 0) ? 1 : 0;
    const size_t smem = static_cast<size_t>(64) * (kpad + 1) * sizeof(float);
    {
        ProfScope ps(LU_PROF_OTHER, s);
        if (fp8) {
            if (int rc_ = smem_attr(quantize_u12_kernel<true>, smem)) return rc_;
            quantize_u12_kernel<true><<<cdiv(N, kScaleTile), 512, smem, s>>>(A, lda, k, w, c0, N, kpad, vec,
                                                                              static_cast<unsigned char*>(Uq), expU);
        } else {
            if (int rc_ = smem_attr(quantize_u12_kernel<false>, smem)) return rc_;
            quantize_u12_kernel<false><<<cdiv(N, 64), 512, smem, s>>>(A, lda, k, w, c0, N, kpad, vec,
                                                                       static_cast<unsigned char*>(Uq), expU);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// A[R0 : R0+M, C0 : C0+N) -= sum_p s_p q(L_p) q(U_p) for the np panels, in
// order.  Panel p's Lq row 0 is operand row ops[p].r0 and its UqT row 0 is
// operand column ops[p].c0.
int schur_tc_apply(float* A, int lda, int R0, int C0, int M, int N, const LowpOperand* ops, int np, bool fp8,
                   int* status, bool leave_sms, cudaStream_t s) {
    if (M <= 0 || N <= 0 || np <= 0) return 0;
    if (np > kTcMaxPanels) return LU_EUNSUPPORTED;
    TcMaps maps;
    TcArgs a{};
    float* C = A + idx(R0, C0, lda);
    a.C = C;
    a.ldc = lda;
    a.M = M;
    a.N = N;
    a.np = np;
    a.status = status;
    a.tma_c = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && (lda & 3) == 0) ? 1 : 0;
    if (a.tma_c) {
        if (int rc = make_c_map(&maps.c, C, lda, M, N)) return rc;
    } else {
        memset(&maps.c, 0, sizeof(maps.c));
    }
    double opbytes = 0.0, kw = 0.0;
    for (int p = 0; p < np; ++p) {
        const LowpOperand& o = ops[p];
        if (int rc = make_operand_map(&maps.op[2 * p], o.Lq, o.Lrows, fp8)) return rc;
        if (int rc = make_operand_map(&maps.op[2 * p + 1], o.Uq, o.Urows, fp8)) return rc;
        a.p[p].rowL = R0 - o.r0;
        a.p[p].rowU = C0 - o.c0;
        a.p[p].nchunk = lowp_kpad(o.w, fp8) / (fp8 ? 128 : 64);
        a.p[p].eLrow = fp8 ? o.eLrow : nullptr;
        a.p[p].eU = fp8 ? o.eU : nullptr;
        opbytes += (fp8 ? 1.0 : 2.0) * (static_cast<double>(M) + N) * lowp_kpad(o.w, fp8);
        kw += o.w;
    }
    const WaitCfg wc = wait_cfg(LU_WAIT_SITE_TC);
    a.wait_ns = wc.wait_ns;
    a.inject = wc.inject;
    const size_t smem = lowp_smem_bytes();
    // The bulk update is HBM-bound; leaving kTsluReserveSMs SMs free lets the
    // next panel's tournament (launched concurrently by the lookahead) run
    // beside it.
    const long long tiles = static_cast<long long>(cdiv(M, kTcBM)) * cdiv(N, kTcBN);
    const int avail = (leave_sms && sm_count() > 2 * kTsluReserveSMs) ? sm_count() - kTsluReserveSMs : sm_count();
    const int grid = static_cast<int>(tiles < avail ? tiles : avail);
    {
        ProfScope ps(LU_PROF_SCHUR_LP, s, 2.0 * M * N * kw, 4.0 * 2.0 * M * N + opbytes);
        if (fp8) {
            if (int rc_ = smem_attr(schur_tc_kernel<true>, smem)) return rc_;
            schur_tc_kernel<true><<<grid, kTcThreads, smem, s>>>(maps, a);
        } else {
            if (int rc_ = smem_attr(schur_tc_kernel<false>, smem)) return rc_;
            schur_tc_kernel<false><<<grid, kTcThreads, smem, s>>>(maps, a);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// Pivot row moves of the deferred panels: rows of each pending Lq (and
// their fp8 exponents) follow the row moves of the step (mv = [count,
// dst[2w], src[2w]] in matrix row positions).  One CTA per (64-byte slice of
// the rows, panel): read every source slice, then write every destination.
__global__ void __launch_bounds__(256) lowp_row_moves_kernel(LowpMoveArgs a, const int* __restrict__ mv, int w) {
    __shared__ uint4 buf[2 * kMaxPanel * 4];
    __shared__ int ebuf[2 * kMaxPanel];
    const int p = blockIdx.y;
    const int cnt = mv[0];
    const int* dst = mv + 1;
    const int* src = mv + 1 + 2 * w;
    uint4* L = reinterpret_cast<uint4*>(a.Lq[p]);
    const int r0 = a.r0[p];
    const int row16 = a.row_bytes / 16;                    // 16-byte words per Lq row
    const int sl = blockIdx.x * 4;                         // this CTA's first 16-byte word of a row
    for (int i = threadIdx.x; i < cnt * 4; i += blockDim.x) {
        const int mvi = i >> 2, wd = sl + (i & 3);
        if (wd < row16) buf[i] = L[static_cast<size_t>(src[mvi] - r0) * (kTcK * a.elem / 16) + wd];
    }
    if (blockIdx.x == 0 && a.eLrow[p])
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) ebuf[i] = a.eLrow[p][src[i] - r0];
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * 4; i += blockDim.x) {
        const int mvi = i >> 2, wd = sl + (i & 3);
        if (wd < row16) L[static_cast<size_t>(dst[mvi] - r0) * (kTcK * a.elem / 16) + wd] = buf[i];
    }
    if (blockIdx.x == 0 && a.eLrow[p])
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) a.eLrow[p][dst[i] - r0] = ebuf[i];
}

int lowp_row_moves(const LowpOperand* ops, int np, bool fp8, const int* mv, int w, cudaStream_t s) {
    if (np <= 0) return 0;
    LowpMoveArgs a{};
    int kpad = 0;
    for (int p = 0; p < np; ++p) {
        a.Lq[p] = const_cast<void*>(ops[p].Lq);
        a.eLrow[p] = fp8 ? const_cast<int*>(ops[p].eLrow) : nullptr;
        a.r0[p] = ops[p].r0;
        kpad = std::max(kpad, lowp_kpad(ops[p].w, fp8));
    }
    a.elem = fp8 ? 1 : 2;
    a.row_bytes = kpad * a.elem;
    {
        ProfScope ps(LU_PROF_PIVOT, s);
        lowp_row_moves_kernel<<<dim3(cdiv(a.row_bytes, 64), np), 256, 0, s>>>(a, mv, w);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

}  // namespace lu
