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
// row of the C tile before waiting for the accumulator).  Every mbarrier wait is
// bounded; a wait that runs out sets an abort flag, the CTA drains and frees
// its tensor memory, and the host sees info = -LU_ETIMEOUT.
#include "common.cuh"
#include "prof.cuh"
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace lu {

constexpr int kTcBM = 128;        // rows of a C tile (MMA M)
constexpr int kTcBN = 128;        // columns of a C tile (MMA N)
constexpr int kTcK = 256;         // padded K of every step (b <= 256)
constexpr int kTcThreads = 192;   // 6 warps
constexpr int kScaleTile = 256;   // operand rows/columns sharing one scale
constexpr long long kWaitLimit = 1ll << 26;   // try_wait polls before giving up
constexpr int kTsluReserveSMs = 16;           // SMs left to the concurrent tournament

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
// Bounded wait for the phase with the given parity.  Returns false on timeout
// or when another role already aborted.
// With check_abort false the wait ignores the abort flag (used to drain
// copies and MMAs still in flight before the CTA exits).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          bool check_abort = true) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (check_abort && (it & 1023) == 1023 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
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

struct TcArgs {
    float* C;          // top-left of the trailing block
    int ldc;
    int M, N;          // trailing block extent handled by this launch
    int col_base;      // global operand column index of C's column 0 (for the U scale index)
    int row_base;      // global operand row index of C's row 0 (for the L scale index)
    const int* expL;   // per 256-row block of Lq: scale exponent (nullptr: scale 1)
    const int* expU;   // per 256-column block of UqT
    int* status;       // set to -LU_ETIMEOUT on a timed-out wait
    int vec4;          // C rows 16-byte aligned (float4 path)
};

template <bool kFp8>
__global__ void __launch_bounds__(kTcThreads, 1) schur_tc_kernel(const __grid_constant__ CUtensorMap tmL,
                                                                 const __grid_constant__ CUtensorMap tmU, TcArgs a) {
    constexpr int kElem = kFp8 ? 1 : 2;
    constexpr int kKBlk = 128 / kElem;                     // K elements per 128-byte row
    constexpr int kNumKBlk = kTcK / kKBlk;                 // 2 (fp8) or 4 (bf16)
    constexpr int kMmaK = 32 / kElem;                      // K per MMA instruction (32 bytes)
    constexpr uint32_t kBlkBytes = 128 * 128;              // one 128-row x 128-byte block
    constexpr uint32_t kTileBytes = kBlkBytes * kNumKBlk;  // A or B tile
    constexpr uint32_t kIdesc = make_idesc<kFp8>();

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB0 = base + kTileBytes;
    unsigned char* sB1 = base + 2 * kTileBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + 3 * kTileBytes);
    uint64_t* a_full = bars + 0;
    uint64_t* a_empty = bars + 1;
    uint64_t* b_full = bars + 2;      // [2]
    uint64_t* b_empty = bars + 4;     // [2]
    uint64_t* acc_full = bars + 6;    // [2]
    uint64_t* acc_empty = bars + 8;   // [2]
    uint64_t* mma_done = bars + 10;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 11);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MB = cdiv(a.M, kTcBM), NB = cdiv(a.N, kTcBN);
    const long long T = static_cast<long long>(MB) * NB;
    const long long t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;

    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_full + i, 1);
            mbar_init(b_empty + i, 1);
            mbar_init(acc_full + i, 1);
            mbar_init(acc_empty + i, 128);
        }
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTcBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int prev_mb = -1, a_uses = 0;
        int issued0 = 0, issued1 = 0;
        for (long long t = t0; t < t1; ++t) {
            const int it = static_cast<int>(t - t0), st = it & 1;
            const int mb = static_cast<int>(t / NB), nb = static_cast<int>(t % NB);
            if (mb != prev_mb) {
                if (prev_mb >= 0 && !mbar_wait(a_empty, (a_uses - 1) & 1, abort_flag)) break;
                mbar_expect_tx(a_full, kTileBytes);
                for (int kb = 0; kb < kNumKBlk; ++kb)
                    tma_load_2d(sA + kb * kBlkBytes, &tmL, kb * kKBlk, mb * kTcBM, a_full);
                prev_mb = mb;
                ++a_uses;
            }
            if (it >= 2 && !mbar_wait(b_empty + st, ((it >> 1) - 1) & 1, abort_flag)) break;
            unsigned char* sB = st ? sB1 : sB0;
            mbar_expect_tx(b_full + st, kTileBytes);
            for (int kb = 0; kb < kNumKBlk; ++kb)
                tma_load_2d(sB + kb * kBlkBytes, &tmU, kb * kKBlk, nb * kTcBN, b_full + st);
            if (st) ++issued1; else ++issued0;
        }
        if (*abort_flag) {      // no CTA exit with TMA writes in flight
            if (a_uses > 0) mbar_wait(a_full, (a_uses - 1) & 1, abort_flag, false);
            if (issued0 > 0) mbar_wait(b_full + 0, (issued0 - 1) & 1, abort_flag, false);
            if (issued1 > 0) mbar_wait(b_full + 1, (issued1 - 1) & 1, abort_flag, false);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int prev_mb = -1, a_uses = 0;
        for (long long t = t0; t < t1; ++t) {
            const int it = static_cast<int>(t - t0), st = it & 1;
            const int mb = static_cast<int>(t / NB);
            if (mb != prev_mb) {
                if (!mbar_wait(a_full, a_uses & 1, abort_flag)) break;
                prev_mb = mb;
                ++a_uses;
            }
            if (!mbar_wait(b_full + st, (it >> 1) & 1, abort_flag)) break;
            if (it >= 2 && !mbar_wait(acc_empty + st, ((it >> 1) - 1) & 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t d = tmem + static_cast<uint32_t>(st * kTcBN);
            const uint32_t aB = smem_u32(sA), bB = smem_u32(st ? sB1 : sB0);
#pragma unroll
            for (int kb = 0; kb < kNumKBlk; ++kb)
#pragma unroll
                for (int kk = 0; kk < kKBlk / kMmaK; ++kk) {
                    const uint32_t off = kb * kBlkBytes + kk * 32;
                    tc_mma<kFp8>(d, sw128_desc(aB + off), sw128_desc(bB + off), kIdesc, (kb | kk) ? 1u : 0u);
                }
            tc_commit(b_empty + st);
            tc_commit(acc_full + st);
            const bool last_of_a = (t + 1 >= t1) || (static_cast<int>((t + 1) / NB) != mb);
            if (last_of_a) tc_commit(a_empty);
        }
        // every MMA issued so far has completed once mma_done flips
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, abort_flag, false);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        for (long long t = t0; t < t1; ++t) {
            const int it = static_cast<int>(t - t0), st = it & 1;
            const int mb = static_cast<int>(t / NB), nb = static_cast<int>(t % NB);
            const int r = mb * kTcBM + q * 32 + lane;
            float* crow = a.C + idx(r < a.M ? r : 0, nb * kTcBN, a.ldc);
            // C does not depend on the accumulator: a full row segment is
            // loaded before the wait, so the tile's 64 KB are in flight
            // while the MMAs run.
            const bool whole = a.vec4 && r < a.M && a.N - nb * kTcBN >= kTcBN;
            float4 cpre[kTcBN / 4];
            if (whole) {
                const float4* p4 = reinterpret_cast<const float4*>(crow);
#pragma unroll
                for (int i = 0; i < kTcBN / 4; ++i) cpre[i] = p4[i];
            }
            if (!mbar_wait(acc_full + st, (it >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            int e = 0;
            if (a.expL) e += a.expL[(a.row_base + mb * kTcBM) / kScaleTile];
            if (a.expU) e += a.expU[(a.col_base + nb * kTcBN) / kScaleTile];
            const float sc = ldexpf(1.0f, e);
#pragma unroll
            for (int c = 0; c < kTcBN; c += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(st * kTcBN + c), v);
                if (r < a.M) {
                    const int cmax = a.N - nb * kTcBN - c;       // valid columns in this chunk
                    if (whole) {
                        float4* p4 = reinterpret_cast<float4*>(crow + c);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float4 x = cpre[c / 4 + i];
                            x.x = fmaf(-sc, v[4 * i + 0], x.x);
                            x.y = fmaf(-sc, v[4 * i + 1], x.y);
                            x.z = fmaf(-sc, v[4 * i + 2], x.z);
                            x.w = fmaf(-sc, v[4 * i + 3], x.w);
                            p4[i] = x;
                        }
                    } else if (a.vec4 && cmax >= 32) {
                        float4* p4 = reinterpret_cast<float4*>(crow + c);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float4 x = p4[i];
                            x.x = fmaf(-sc, v[4 * i + 0], x.x);
                            x.y = fmaf(-sc, v[4 * i + 1], x.y);
                            x.z = fmaf(-sc, v[4 * i + 2], x.z);
                            x.w = fmaf(-sc, v[4 * i + 3], x.w);
                            p4[i] = x;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (i < cmax) crow[c + i] = fmaf(-sc, v[i], crow[c + i]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty + st);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcBN));
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

// One CTA per 256-row block of L21 = A[r0 + 256 blk .., k : k+w).  Lq is
// [M x 256] with K padded by zeros.
template <bool kFp8>
__global__ void __launch_bounds__(256) quantize_l21_kernel(const float* __restrict__ A, int lda, int r0, int M, int k,
                                                           int w, unsigned char* __restrict__ Lq, int* __restrict__ expL) {
    __shared__ float red[32];
    const int rb = blockIdx.x * kScaleTile;
    const int nr = min(kScaleTile, M - rb);
    int e = 0;
    if (kFp8) {
        float mx = 0.0f;
        for (int i = threadIdx.x; i < nr * w; i += blockDim.x) mx = fmaxf(mx, fabsf(A[idx(r0 + rb + i / w, k + i % w, lda)]));
        mx = block_max(mx, red);
        e = fp8_exponent(mx);
        if (threadIdx.x == 0) expL[blockIdx.x] = e;
    }
    for (int i = threadIdx.x; i < nr * kTcK; i += blockDim.x) {
        const int rr = i / kTcK, kk = i % kTcK;
        const float x = kk < w ? A[idx(r0 + rb + rr, k + kk, lda)] : 0.0f;
        store_q<kFp8>(Lq, static_cast<size_t>(rb + rr) * kTcK + kk, kFp8 ? ldexpf(x, -e) : x);
    }
}

// One CTA per 256-column block of U12 = A[k : k+w, c0 + 256 blk ..).  UqT is
// [N x 256] (transposed: K-major), K padded by zeros.
template <bool kFp8>
__global__ void __launch_bounds__(256) quantize_u12_kernel(const float* __restrict__ A, int lda, int k, int w, int c0,
                                                           int N, unsigned char* __restrict__ Uq, int* __restrict__ expU) {
    __shared__ float red[32];
    __shared__ float tile[32][kTcK + 1];
    const int cb = blockIdx.x * kScaleTile;
    const int nc = min(kScaleTile, N - cb);
    int e = 0;
    if (kFp8) {
        float mx = 0.0f;
        for (int i = threadIdx.x; i < w * nc; i += blockDim.x) mx = fmaxf(mx, fabsf(A[idx(k + i / nc, c0 + cb + i % nc, lda)]));
        mx = block_max(mx, red);
        e = fp8_exponent(mx);
        if (threadIdx.x == 0) expU[blockIdx.x] = e;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int cc = 0; cc < nc; cc += 32) {
        // read 32 columns x w rows (coalesced along columns), transpose in smem
        for (int kk = warp; kk < kTcK; kk += 8)
            tile[lane][kk] = (kk < w && cc + lane < nc) ? A[idx(k + kk, c0 + cb + cc + lane, lda)] : 0.0f;
        __syncthreads();
        for (int i = threadIdx.x; i < 32 * kTcK; i += blockDim.x) {
            const int col = i / kTcK, kk = i % kTcK;
            if (cc + col < nc) {
                const float x = tile[col][kk];
                store_q<kFp8>(Uq, static_cast<size_t>(cb + cc + col) * kTcK + kk, kFp8 ? ldexpf(x, -e) : x);
            }
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
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kTcK), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kTcK) * elem};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem), 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
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

size_t lowp_smem_bytes(bool fp8) {
    const size_t tile = 128 * 128 * (fp8 ? 2 : 4);
    return 1024 + 3 * tile + 128;
}

int quantize_l21(const float* A, int lda, int m, int k, int w, bool fp8, void* Lq, int* expL, cudaStream_t s) {
    const int r0 = k + w, M = m - r0;
    if (M <= 0) return 0;
    {
        ProfScope ps(LU_PROF_OTHER, s);
        if (fp8)
            quantize_l21_kernel<true><<<cdiv(M, kScaleTile), 256, 0, s>>>(A, lda, r0, M, k, w,
                                                                           static_cast<unsigned char*>(Lq), expL);
        else
            quantize_l21_kernel<false><<<cdiv(M, kScaleTile), 256, 0, s>>>(A, lda, r0, M, k, w,
                                                                            static_cast<unsigned char*>(Lq), expL);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

int quantize_u12(const float* A, int lda, int k, int w, int c0, int c1, bool fp8, void* Uq, int* expU,
                 cudaStream_t s) {
    const int N = c1 - c0;
    if (N <= 0) return 0;
    {
        ProfScope ps(LU_PROF_OTHER, s);
        if (fp8)
            quantize_u12_kernel<true><<<cdiv(N, kScaleTile), 256, 0, s>>>(A, lda, k, w, c0, N,
                                                                           static_cast<unsigned char*>(Uq), expU);
        else
            quantize_u12_kernel<false><<<cdiv(N, kScaleTile), 256, 0, s>>>(A, lda, k, w, c0, N,
                                                                            static_cast<unsigned char*>(Uq), expU);
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

// C[0:M, 0:N) -= scale * Lq[0:M] . Uq[0:N]^T.  Lq has M rows, Uq has N rows
// (both 256 wide); row_base / col_base index the scale arrays.
int schur_tc(float* C, int ldc, int M, int N, const void* Lq, const void* Uq, const int* expL, const int* expU,
             int row_base, int col_base, bool fp8, int* status, int w, cudaStream_t s) {
    if (M <= 0 || N <= 0) return 0;
    CUtensorMap tmL, tmU;
    if (int rc = make_operand_map(&tmL, Lq, M, fp8)) return rc;
    if (int rc = make_operand_map(&tmU, Uq, N, fp8)) return rc;
    TcArgs a{};
    a.C = C;
    a.ldc = ldc;
    a.M = M;
    a.N = N;
    a.col_base = col_base;
    a.row_base = row_base;
    a.expL = fp8 ? expL : nullptr;
    a.expU = fp8 ? expU : nullptr;
    a.status = status;
    a.vec4 = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && (ldc & 3) == 0) ? 1 : 0;
    const size_t smem = lowp_smem_bytes(fp8);
    // The update is HBM-bound; leaving kTsluReserveSMs SMs free lets the next
    // panel's tournament (launched concurrently by the lookahead) run beside it.
    const long long tiles = static_cast<long long>(cdiv(M, kTcBM)) * cdiv(N, kTcBN);
    const int avail = sm_count() > 2 * kTsluReserveSMs ? sm_count() - kTsluReserveSMs : sm_count();
    const int grid = static_cast<int>(tiles < avail ? tiles : avail);
    {
        ProfScope ps(LU_PROF_SCHUR_LP, s, 2.0 * M * N * w, 4.0 * 2.0 * M * N + (fp8 ? 1.0 : 2.0) * (M + N) * kTcK);
        if (fp8) {
            if (int rc_ = smem_attr(schur_tc_kernel<true>, smem)) return rc_;
            schur_tc_kernel<true><<<grid, kTcThreads, smem, s>>>(tmL, tmU, a);
        } else {
            if (int rc_ = smem_attr(schur_tc_kernel<false>, smem)) return rc_;
            schur_tc_kernel<false><<<grid, kTcThreads, smem, s>>>(tmL, tmU, a);
        }
        count_launches(1);
    }
    LU_LAUNCHED();
    return 0;
}

}  // namespace lu
