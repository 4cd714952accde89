// Internal helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include "../../include/conflux_lu.h"
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#define LU_TRY(expr)                                                  \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) return LU_ELAUNCH;                     \
    } while (0)

#define LU_LAUNCHED()                                                 \
    do {                                                              \
        if (cudaPeekAtLastError() != cudaSuccess) {                   \
            cudaGetLastError();                                       \
            return LU_ELAUNCH;                                        \
        }                                                             \
    } while (0)

namespace lu {

// Stream-ordered device allocation from the library's own memory pool (one
// per device, created on first use): freed memory stays reserved for reuse
// up to 16 GB instead of going back to the driver at every synchronize, so
// repeated calls do not re-map their workspace; the caller's default pool
// is left alone.  Same contract as cudaMallocAsync; free with cudaFreeAsync.
cudaError_t lu_malloc_async(void** p, size_t bytes, cudaStream_t s);

// 16-byte asynchronous copy global -> shared (cp.async); bytes < 16 reads
// that many and zero-fills the rest (0: nothing is read).  Both addresses
// 16-byte aligned.  cp_async_wait_all() waits for the thread's own copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most one committed group of the thread's copies is pending
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Raise a kernel's dynamic shared-memory cap to at least `bytes` (per kernel
// and device; never lowered, so concurrent callers with different sizes on
// other host threads cannot shrink it under each other).
template <typename K>
inline int smem_attr(K* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LU_ELAUNCH;
    }
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = done[std::make_pair(reinterpret_cast<const void*>(kernel), dev)];
    if (cur >= bytes) return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) !=
        cudaSuccess) {
        cudaGetLastError();
        return LU_ELAUNCH;
    }
    cur = bytes;
    return 0;
}

// Bounded device waits.  Every spin or mbarrier wait of the library gives up
// after a wall-clock deadline read from %globaltimer (nanoseconds), not
// after a poll count: a poll may suspend for a hardware-defined time, so a
// count bounds nothing.  A wait that runs out records an error status that
// the host turns into LU_ETIMEOUT, and the kernel exits normally.
constexpr unsigned long long kWaitDefaultNs = 4000000000ull;   // dependency waits: 4 s
constexpr unsigned long long kDrainWaitNs = 4000000000ull;     // waits for the kernel's own copies in flight

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per wait site: the deadline of its dependency waits and whether a test has
// asked it to wait once on something nothing will ever signal (the way the
// tests make a wait run out without a fault).  Process-wide; set only by
// lu_test_wait_config.
struct WaitCfg {
    unsigned long long wait_ns;
    int inject;
};
WaitCfg wait_cfg(int site);     // site: LU_WAIT_SITE_*

constexpr int kMaxPanel = 256;          // largest supported panel width b
constexpr int kTsluThreads = 256;       // threads per tournament CTA
constexpr int kTsluMaxCluster = 8;      // portable cluster size

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline size_t idx(int i, int j, int ld) {
    return static_cast<size_t>(i) * static_cast<size_t>(ld) + static_cast<size_t>(j);
}

// Tournament geometry of one step: rows [k, m), panel [k, k+w).
struct TsluShape {
    int H;        // rows of a first-level node (a "super-leaf")
    int nsuper;   // number of first-level nodes
    int nr_max;   // most rows any node stacks
    int C;        // CTAs per node (cluster size)
    int R;        // rows per CTA
    int ws;       // row stride of the node's rows in shared memory (elements)
    int blocked;  // node GEPP: 1 blocked on one CTA, 2 blocked over a cluster, 0 column by column
    size_t smem;  // dynamic shared memory per CTA (bytes)
};

// Largest dynamic shared memory a tournament CTA may take (the kernel also
// uses up to ~6 KB of static shared memory).
constexpr size_t kTsluSmemLimit = 232448 - 8192;

// Leaves of h rows whose selection keeps every row (h <= w) are merged
// upward until a node holds more than w rows: selection is independent of
// the order in which candidate rows are stacked, so a node made only of
// such leaves selects from its whole contiguous row range.
TsluShape tslu_shape(int m, int k, int w, int h, int max_cluster, int elem);
int tslu_max_cluster();

// Host entry points of the factorization pieces (stream-ordered, no sync).
template <typename T>
int tslu_select(const T* A, int lda, int m, int k, int w, int h, int* lists, int* counts, size_t list_stride_nodes,
                T* a00, int* info, const int** root_list, cudaStream_t s);
template <typename T>
int pivot_apply(T* A, int lda, int m, int n, int k, int w, const int* root_list, const T* a00, int* piv, int* mv,
                cudaStream_t s);
// L21 = A21 * U^{-1} with U the upper triangle of a w x w block (stride ldu)
template <typename T>
int trsm_l21(T* A, int lda, int m, int k, int w, const T* U, int ldu, cudaStream_t s);
template <typename T>
int trsm_u12(T* A, int lda, int n, int k, int w, cudaStream_t s);
// A[r0:m, c0:c1) -= A[r0:m, k:k+w) * A[k:k+w, c0:c1)   (r0 = k + w)
int schur_f64(double* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s);
int schur_f32(float* A, int lda, int m, int k, int w, int c0, int c1, cudaStream_t s);
// Cholesky pieces (csrc/chol.cu, csrc/schur_f64.cu)
constexpr int kCholMaxPanel = 128;      // largest Cholesky panel width
// lower triangle of rows [c0, n) x columns [c0, c1) -= A[:, k:k+w) A[:, k:k+w)^T
template <typename T>
int syrk_lower(T* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s);
template <>
int syrk_lower<double>(double* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s);   // schur_f64.cu
template <>
int syrk_lower<float>(float* A, int lda, int n, int k, int w, int c0, int c1, cudaStream_t s);     // schur_f32.cu
int getrs_f64(int n, int nrhs, const double* LU, int lda, const int* piv, double* B, int ldb, cudaStream_t s);

// What a solve needs besides B (csrc/getrs.cu): the composed row permutation
// and the transposed inverses of the diagonal blocks of L and U.
template <typename T>
struct SolvePlan {
    int n = 0;
    const T* LU = nullptr;
    int lda = 0;
    int* perm = nullptr;
    T* DT = nullptr;           // inverses of the diagonal blocks, [block][L, U][NB][NB] row-major
    T* M = nullptr;            // coupling blocks inv(L_bb) L_{b,b-1} / inv(U_bb) U_{b,b+1}, same layout
    int* off = nullptr;        // work items before each block step
    int chol = 0;              // LU is a Cholesky factor L: U = L^T, no permutation
};
template <typename T>
int solve_plan_make(int n, const T* LU, int lda, const int* piv, SolvePlan<T>* p, cudaStream_t s);
template <typename T>
int solve_plan_apply(const SolvePlan<T>& p, int nrhs, T* B, int ldb, cudaStream_t s);
template <typename T>
void solve_plan_free(SolvePlan<T>* p, cudaStream_t s);
int getrs_f32(int n, int nrhs, const float* LU, int lda, const int* piv, float* B, int ldb, cudaStream_t s);

// Factorization + refinement pieces of the solver (csrc/ir.cu), shared with
// the serving runtime.
struct IrFactors {
    int n = 0;
    float* A32 = nullptr;      // binary32 factors
    int* piv = nullptr;
    int* info = nullptr;
    int precision = 0;         // LU_PREC_* of the factors
    SolvePlan<float> plan;     // solve plan of these factors
};
int ir_factor(int n, const double* A, int lda, int prec, int b, int h, IrFactors* f, cudaStream_t s);
int ir_refine(IrFactors* f, const double* A, int lda, int nrhs, const double* B, int ldb, double* X, int ldx,
              const ir_opts* o, ir_result* res, cudaStream_t s);
void ir_release(IrFactors* f, cudaStream_t s);
size_t ir_workspace_bytes(int n, int nrhs, int restart);

// One request of a shared (batched) solve launch (csrc/serve_batch.cu).
// Device pointers; n <= 1024, 1 <= nrhs <= 64.
struct BatchReq {
    const double* A;           // binary64 matrix (lda)
    const double* B;           // right-hand sides (ldb)
    double* X;                 // solution, n x nrhs (ld nrhs)
    double* R;                 // residual, n x nrhs (ld nrhs)
    float* r;                  // binary32 correction, n x nrhs (ld nrhs)
    float* F;                  // binary32 factors, n x n (ld n)
    int* piv;                  // their pivots
    double* cw;                // 2 * nrhs scratch: max|b_c|, then max|r_c|
    double anorm;              // ||A||_inf (set by the launch)
    int lda, ldb, n, nrhs;
    int factor;                // 1: F is copied from A and factored here; 0: F holds cached factors
    int pad;
};
int batch_solve(std::vector<BatchReq>& reqs, const std::vector<double>& tol, int max_iter, std::vector<int>& out,
                std::vector<int>& iters, std::vector<double>& eta, cudaStream_t s);

// Low-precision tensor-core Schur update (csrc/schur_lowp.cu).
constexpr int kLowpK = 256;     // operand rows are 256 K-elements wide (padded)
constexpr int kTcMaxPanels = 4; // pending panels one update launch applies
constexpr int kDeferDefault = 4;   // pending panels of the bf16 / fp8 factorization by default
// One quantized panel: Lq (rows from the step's first trailing row r0,
// K-major, kLowpK wide) with per-row fp8 exponents, and UqT (rows = the
// trailing columns from c0) with one fp8 exponent per 256 rows.
struct LowpOperand {
    const void* Lq;
    int Lrows;
    const int* eLrow;
    const void* Uq;
    int Urows;
    const int* eU;
    int r0, c0, w;
};
struct LowpMoveArgs {
    void* Lq[kTcMaxPanels];
    int* eLrow[kTcMaxPanels];
    int r0[kTcMaxPanels];
    int elem, row_bytes;
};
size_t lowp_smem_bytes();
int lowp_kpad(int w, bool fp8);
int quantize_l21(const float* A, int lda, int m, int k, int w, bool fp8, void* Lq, int* eLrow, cudaStream_t s);
int quantize_u12(const float* A, int lda, int k, int w, int c0, int c1, bool fp8, void* Uq, int* expU, cudaStream_t s);
// A[R0:R0+M, C0:C0+N) -= sum_p s_p q(L_p) q(U_p), panels in order
int schur_tc_apply(float* A, int lda, int R0, int C0, int M, int N, const LowpOperand* ops, int np, bool fp8,
                   int* status, bool leave_sms, cudaStream_t s);
// the step's row moves (pivot_apply's move list) applied to pending Lq rows
int lowp_row_moves(const LowpOperand* ops, int np, bool fp8, const int* mv, int w, cudaStream_t s);

}  // namespace lu
