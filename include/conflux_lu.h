/*
 * conflux_lu.h -- C ABI of the GB300 tournament-pivoting LU library (and
 * of its Cholesky variant).
 *
 * The operations follow the paper's statement of the problem: in-place
 * PA = LU of a dense matrix (Fig. 1; Algorithm 1, where A_t shrinks by v
 * columns and the chosen rows each step), computed as a blocked right-looking
 * LU whose v pivot rows per step come from tournament pivoting (Section 7.3)
 * and whose block updates are the triangular solves FactorizeA10 /
 * FactorizeA01 and the Schur update FactorizeA11 (Section 7.2).  Everything
 * else follows LAPACK getrf/getrs conventions.
 *
 * Layout.  Matrices are ROW-MAJOR: element (i, j) of A sits at A[i*lda + j],
 * lda >= max(1, columns).  Row swaps are then contiguous copies, and this is
 * PyTorch's native layout.
 *
 * Ownership.  Matrix, vector, pivot and info pointers are DEVICE pointers
 * owned by the caller, unless an argument says "host".  The library keeps no
 * pointer past the work it enqueues on the given stream.  Internal workspace
 * is taken stream-ordered (cudaMallocFromPoolAsync) from a memory pool the
 * library creates per device and returned on the same stream; the pool
 * keeps up to 16 GB of freed memory reserved for the next calls, and the
 * caller's default pool is not touched.
 *
 * Asynchrony.  Every call validates its arguments on the host, enqueues its
 * work on `stream` and returns; results are ready when the stream reaches
 * that point.  Calls on one stream are ordered; calls that share buffers on
 * different streams must be ordered by the caller.
 *
 * Status.  The return value is
 *     0                       enqueued,
 *    -i  (i >= 1)             argument i is invalid (checked before any work),
 *     LU_E* (positive)        a runtime failure (see below).
 * Numerical status goes to a caller-provided DEVICE int `info`:
 *     0       success,
 *     j + 1   U(j, j) is exactly zero for the first such j.  The factorization
 *             still completes (as getrf); the L column below a zero pivot is
 *             set to zero instead of dividing by zero.
 * Inputs are assumed finite; results on NaN/Inf inputs are unspecified.
 */
#ifndef CONFLUX_LU_H
#define CONFLUX_LU_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runtime failure codes (positive return values). */
#define LU_ENOMEM       1   /* workspace allocation failed                    */
#define LU_ELAUNCH      2   /* a kernel launch or CUDA call failed            */
#define LU_ETIMEOUT     3   /* a bounded device-side wait ran out             */
#define LU_EBUSY        4   /* serving: no slot or HBM budget left            */
#define LU_EUNSUPPORTED 5   /* valid but unsupported combination of options   */
#define LU_ENOTFOUND    6   /* serving: unknown ticket                        */

/* Arithmetic of the factorization. */
typedef enum {
    LU_PREC_F64 = 0,        /* every step in binary64                          */
    LU_PREC_F32 = 1,        /* every step in binary32                          */
    LU_PREC_BF16 = 2,       /* binary32 panel and solves; Schur update with
                               bfloat16 operands, fp32 accumulation            */
    LU_PREC_FP8 = 3         /* as BF16 but fp8 e4m3 operands with one
                               power-of-two scale per 256 x 256 tile           */
} lu_precision;

/* Options of the blocked factorization.  Zero fields take defaults. */
typedef struct {
    int b;                  /* panel width v (Section 7.2 "Blocking parameter
                               v"); default 256 for n >= 4096, else 32        */
    int h;                  /* tournament leaf height: rows per leaf of the
                               first round (Section 7.3); default 128          */
    int precision;          /* lu_precision; default LU_PREC_F64               */
    int defer;              /* BF16 / FP8 factorization only: panels whose
                               trailing updates are held back and applied in
                               one pass over the trailing matrix (1..4;
                               0 = 4); the factors do not depend on it       */
    int reserved[4];        /* must be zero                                     */
} lu_opts;

/*
 * lu_factor -- in-place PA = LU of an n x n matrix (Algorithm 1).
 *   n      order, n >= 0
 *   A      device, n x n row-major, lda >= max(1, n); overwritten by L (unit
 *          lower, diagonal not stored) and U
 *   lda    leading dimension (elements)
 *   piv    device int[n]; piv[i] = the 0-based row that was swapped with row
 *          i at step i (LAPACK ipiv, 0-based)
 *   info   device int; see "Status"
 *   stream CUDA stream (0 = legacy default stream)
 * Uses b = 256 (n >= 4096) or 32, h = 128, binary64 throughout.
 */
int lu_factor(int n, double *A, int lda, int *piv, int *info, cudaStream_t stream);

/*
 * lu_factor_ex -- rectangular m x n factorization with options.  min(m, n)
 * pivots are produced; for m < n the result is L (m x m) and an upper
 * trapezoidal U (m x n).  opts may be NULL (defaults).  Only LU_PREC_F64 is
 * accepted here; the binary32 and mixed-precision factorizations are
 * lu_factor_f32 with opts->precision F32, BF16 or FP8.
 * Tournament nodes hold up to max(leaf rows, 2b) x b panel values in the
 * shared memory of one thread-block cluster: b <= 256 and
 * max(h', 2b) * b <= 204800 where h' is the first tree level's row count.
 */
int lu_factor_ex(int m, int n, double *A, int lda, int *piv, int *info,
                 const lu_opts *opts, cudaStream_t stream);

/*
 * lu_memory_pool -- the memory pool (a cudaMemPool_t) from which the library
 * takes its stream-ordered workspace on the current device, created on first
 * use with a release threshold of 16 GB: for inspection
 * (cudaMemPoolGetAttribute) or trimming (cudaMemPoolTrimTo) by the caller.
 * Returns -1 for a null pointer, LU_ELAUNCH if the pool cannot be created.
 */
int lu_memory_pool(void **pool);

/*
 * lu_factor_host -- lu_factor_ex on a matrix in HOST memory: the call copies
 * A to the device, factors it there (Algorithm 1, binary64) and copies L\U,
 * the pivots and info back, then returns with the results in host memory
 * (it synchronizes `stream`).
 *   m, n, lda, opts  as lu_factor_ex (opts->precision must be 0 or F64)
 *   A     HOST, m x n row-major; overwritten by L and U.  Page-locked memory
 *         (cudaHostAlloc / cudaHostRegister) lets the copies run at the
 *         link's rate, and each step's b finished rows then go back while
 *         the later steps run; pageable memory works, more slowly, and gets
 *         all of L\U back after the last step.
 *   piv   HOST int[min(m, n)]
 *   info  HOST int
 * Device memory: one m x n binary64 buffer plus the factorization's
 * workspace, taken from the stream-ordered allocator and returned before the
 * call returns.  Returns 0, -i for an invalid argument i, LU_ENOMEM,
 * LU_ELAUNCH, or LU_EUNSUPPORTED for a precision other than binary64.
 */
int lu_factor_host(int m, int n, double *A, int lda, int *piv, int *info,
                   const lu_opts *opts, cudaStream_t stream);

/*
 * lu_solve -- X = U^{-1} L^{-1} P B with the factors of lu_factor: the
 * linear-system solve that the factorization exists for (the paper names
 * linear solvers as LU's use in Section 1 and does not spell the solve out;
 * this is LAPACK getrs's forward and backward substitution).
 *   n, LU, lda, piv  as returned by lu_factor (device)
 *   nrhs  number of right-hand sides, 0 <= nrhs <= 384
 *   B     device, n x nrhs row-major, ldb >= max(1, nrhs); overwritten by X
 * Returns 0, -i for an invalid argument i, or LU_ENOMEM / LU_ELAUNCH /
 * LU_ETIMEOUT (a bounded device wait ran out; B is then invalid).
 */
int lu_solve(int n, int nrhs, const double *LU, int lda, const int *piv,
             double *B, int ldb, cudaStream_t stream);


/*
 * lu_factor_f32 -- the same factorization on a binary32 matrix.
 * opts->precision selects the Schur-update arithmetic:
 *   LU_PREC_F32 (default)  binary32 everywhere;
 *   LU_PREC_BF16 / FP8     binary32 panel, pivoting and triangular solves;
 *                          the trailing update takes bfloat16 / fp8-e4m3
 *                          operands (fp8: one power-of-two scale per 256 x 256
 *                          operand tile) with fp32 accumulation on the
 *                          tensor cores.  Needs m == n and b a multiple of
 *                          128 (else LU_EUNSUPPORTED).
 * A negative *info (-LU_ETIMEOUT) reports a device-side wait that ran out;
 * the factors are then invalid.
 */
int lu_factor_f32(int m, int n, float *A, int lda, int *piv, int *info,
                  const lu_opts *opts, cudaStream_t stream);

/* lu_solve_f32 -- X = U^{-1} L^{-1} P B with binary32 factors (B overwritten). */
int lu_solve_f32(int n, int nrhs, const float *LU, int lda, const int *piv,
                 float *B, int ldb, cudaStream_t stream);

/*
 * chol_factor -- in-place Cholesky factorization A = L L^T of a symmetric
 * positive definite n x n matrix, binary64 (the kernel that Section 2.2 and
 * the Conclusions name for the same schedule; Algorithm 1's blocked
 * right-looking loop without TournPivot: per step of width b, factor the
 * diagonal block, solve the panel L21 = A21 L00^{-T}, update the lower
 * triangle of the trailing matrix).
 *   n      order, n >= 0
 *   A      device, n x n row-major, lda >= max(1, n).  Only the lower
 *          triangle (j <= i) is read; on return it holds L.  The strict
 *          upper triangle is not referenced.
 *   info   device int: 0, or j + 1 for the first column j whose pivot is not
 *          positive (or is NaN).  The factorization is then incomplete:
 *          columns before j hold L, later ones are unspecified (finite or
 *          not; no device fault).
 *   opts   may be NULL.  opts->b: panel width, 1..128 (default 128 for
 *          n >= 4096, else 64); opts->h must be 0; opts->precision must be
 *          0 or LU_PREC_F64.
 * Every element receives its update terms in ascending column order as one
 * fused multiply-add each, then its square root (diagonal) or one IEEE
 * division, so the result does not depend on b.
 * Returns 0, -i for an invalid argument i (1 n, 2 A, 3 lda, 4 info,
 * 5 opts), or LU_ENOMEM / LU_ELAUNCH.
 */
int chol_factor(int n, double *A, int lda, int *info, const lu_opts *opts,
                cudaStream_t stream);

/* chol_factor_f32 -- the same factorization in binary32 (opts->precision 0
 * or LU_PREC_F32). */
int chol_factor_f32(int n, float *A, int lda, int *info, const lu_opts *opts,
                    cudaStream_t stream);

/*
 * chol_solve -- X = L^{-T} L^{-1} B with the factor of chol_factor.
 *   n, L, lda  as returned by chol_factor (device; lower triangle read)
 *   nrhs  number of right-hand sides, 0 <= nrhs <= 384
 *   B     device, n x nrhs row-major, ldb >= max(1, nrhs); overwritten by X
 * Blocked forward and backward substitution (the LU solve's work list with
 * U = L^T and no permutation).  Returns 0, -i for an invalid argument i
 * (1 n, 2 nrhs, 3 L, 4 lda, 5 B, 6 ldb), or LU_ENOMEM / LU_ELAUNCH /
 * LU_ETIMEOUT (a bounded device wait ran out).
 */
int chol_solve(int n, int nrhs, const double *L, int lda, double *B, int ldb,
               cudaStream_t stream);
/* chol_solve_f32 -- the same with a binary32 factor. */
int chol_solve_f32(int n, int nrhs, const float *L, int lda, float *B, int ldb,
                   cudaStream_t stream);

/*
 * lu_gemm_lowp -- the low-precision Schur update on its own:
 *   C -= sL * sU * round(L / sL) * round(U / sU)
 * L: M x K (ldl), U: K x N (ldu), C: M x N (ldc), all binary32 device
 * arrays, K <= 256.  round = bfloat16 (precision LU_PREC_BF16, scales 1) or
 * fp8 e4m3 with saturation (LU_PREC_FP8; sL per 256 rows of L, sU per 256
 * columns of U, each the smallest power of two with max|block| / s <= 448).
 * Products accumulate in fp32 on the tensor cores.  status (device int) is
 * 0, or -LU_ETIMEOUT if a device-side wait ran out.
 */
int lu_gemm_lowp(int M, int N, int K, const float *L, int ldl, const float *U,
                 int ldu, float *C, int ldc, int precision, int *status,
                 cudaStream_t stream);

/*
 * lu_residual -- R = B - A X in binary64 and, per column c, the normwise
 * backward error eta[c] = ||r_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf).
 * A: n x n (lda); X, B, R: n x nrhs (ldx, ldb, ldr); eta: device double[nrhs].
 */
int lu_residual(int n, int nrhs, const double *A, int lda, const double *X,
                int ldx, const double *B, int ldb, double *R, int ldr,
                double *eta, cudaStream_t stream);

/*
 * lu_residual_noalloc -- lu_residual for callers that must not allocate
 * device memory while they run: a serving loop that reserves all of its
 * memory before taking requests (so that no request can fail halfway on an
 * out-of-memory), or a process in which another framework's caching
 * allocator owns the GPU's memory.  The paper has no counterpart; this is a
 * deployment variant of the residual and backward-error computation.
 *
 * Same arguments, results and layouts as lu_residual, with nrhs <= 64
 * (larger nrhs returns -2 before any work).  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its reduction scratch is one fixed
 * array of about 160 KB per device, placed in the library and kept until the
 * process exits.  Each call looks up that array's device address
 * (cudaGetSymbolAddress) with the device current, so a device reset between
 * calls leaves no stale address behind; the first call on a device may load
 * the library's device code, so make it before any stream capture.  Every call on a device uses the same
 * array, so calls whose work overlaps on the GPU (different streams, no
 * ordering between them) race and give wrong results; calls ordered on one
 * stream are safe.  Nothing in the array has to start at zero: each call
 * writes every slot it reads.
 */
int lu_residual_noalloc(int n, int nrhs, const double *A, int lda,
                        const double *X, int ldx, const double *B, int ldb,
                        double *R, int ldr, double *eta, cudaStream_t stream);

/*
 * lu_factor_batched -- factor `batch` independent square matrices in one
 * persistent launch: Algorithm 1 (TournPivot of Section 7.3, then
 * FactorizeA10 / A01 / A11 of Section 7.2) run per matrix by one CTA, the
 * largest matrices scheduled first.  Each matrix's pivots and factors are
 * those of lu_factor_ex with the same b and h, whatever else is in the
 * batch.
 *   n, lda  device int[batch]: order (0 <= n <= 1024) and leading dimension
 *   A       device array of batch device pointers (double* or float*)
 *   piv     device array of batch device pointers to int[n]
 *   info    device int[batch]: as lu_factor's info, or -1 when n is out of
 *           range, a pointer is null or lda < n (that matrix is skipped)
 *   dtype   LU_PREC_F64 or LU_PREC_F32
 * Panel width b = lu_batched_panel_width_dt(n, dtype), leaf height h = 128.
 */
int lu_factor_batched(int batch, const int *n, void *const *A, const int *lda,
                      int *const *piv, int *info, int dtype, cudaStream_t stream);

/* Panel width the batched factorization uses for an n x n binary64 matrix
 * (lu_batched_panel_width) or for dtype LU_PREC_F64 / LU_PREC_F32
 * (lu_batched_panel_width_dt; -2 for another dtype).  The width comes from a
 * table over six size classes (n <= 32, <= 64, <= 128, <= 256, <= 512,
 * <= 1024) whose defaults were measured on GB300. */
int lu_batched_panel_width(int n);
int lu_batched_panel_width_dt(int n, int dtype);

/* Replace the size-class table of one dtype (count = 6 widths in 1..32) for
 * the batched factorizations launched after the call, process-wide (a tuning
 * sweep); widths = NULL restores the measured defaults.  Returns 0, -1 bad
 * dtype, -2 a width out of range, -3 count != 6. */
int lu_batched_set_panel_widths(int dtype, const int *widths, int count);

/*
 * lu_solve_batched -- X = U^{-1} L^{-1} P B for each matrix of a batched
 * factorization, one launch.  n, nrhs (1..8), lda, ldb: device int[batch];
 * LU, piv, B: device arrays of device pointers.  B is overwritten.
 */
int lu_solve_batched(int batch, const int *n, const int *nrhs, void *const *LU,
                     const int *lda, int *const *piv, void *const *B,
                     const int *ldb, int dtype, cudaStream_t stream);

/* Options and result of ir_solve.  Zero fields take defaults. */
typedef struct {
    int precision;          /* first factorization: LU_PREC_BF16 (also when 0),
                               LU_PREC_FP8 or LU_PREC_F32                      */
    int b, h;               /* panel width and leaf height (defaults 128/128) */
    double tol;             /* stop when max_c eta_c <= tol (default 1e-12)    */
    int max_iter;           /* outer refinement steps (default 40)             */
    int gmres_restart;      /* FGMRES restart length (default 30, max 200)     */
    int krylov_products;    /* products A z inside FGMRES: 0 (default) binary32
                               multiplies first, binary64 from the first cycle
                               that cuts eta by less than 10x; 1 binary64
                               only; 2 binary32 multiplies only               */
    int inner_steps;        /* binary32-product inner steps per classical step
                               (0: default 3; negative: none)                  */
    int reserved[2];        /* must be zero                                     */
} ir_opts;

typedef struct {
    int iters;              /* outer refinement steps taken                    */
    int gmres_iters;        /* inner FGMRES iterations in total                */
    int path;               /* 0: classical refinement converged; 1: FGMRES-IR
                               converged; -1: tol not reached                  */
    int info;               /* info of the factorization                        */
    double eta;             /* final max_c eta_c                                */
    double eta0;            /* max_c eta_c of the first solve                   */
    int precision;          /* factorization precision in use at the end        */
    int refactors;          /* times the ladder moved up a precision            */
    int cycles32;           /* FGMRES cycles run with binary32-multiply products */
    int cycles64;           /* FGMRES cycles run with binary64 products          */
    int inner_steps;        /* binary32-product inner steps of classical steps   */
} ir_result;

/*
 * ir_solve -- solve A X = B to binary64 backward error tol with a
 * low-precision factorization and binary64 refinement.  A (n x n, lda) and
 * B (n x nrhs, ldb) are read only; X (n x nrhs, ldx) receives the solution;
 * all three are device arrays.  res is a HOST pointer.  The refinement
 * decides on the host when to stop, so this call synchronizes `stream` and
 * returns when X is final.  Classical refinement runs while each step cuts
 * eta by 4x or more: from the binary64 residual r it solves A d = r with up
 * to inner_steps binary32-product steps (d += LU^{-1} (r - A d), A d with
 * binary32 multiplies, stopping once the inner residual stops shrinking by
 * 2x or falls below 1e-6 |r|), then x += d.  After that the correction equation is
 * solved by right-preconditioned flexible GMRES (binary64 Arnoldi and
 * Gram-Schmidt, the fp32 LU solve as preconditioner).  Its products A z
 * first use binary32 multiplies (A and z rounded to binary32, 32-term
 * binary32 runs summed in binary64) with an inner tolerance of 1e-6: the
 * outer binary64 residual corrects what they miss.  Once such a cycle cuts
 * eta by less than 10x the products are binary64 (kappa too large for
 * them), unless the factors are fp8: those are refactored in bf16 first and
 * the binary32 products kept.  When a binary64 FGMRES cycle
 * gains less than 10x, or two cycles do not reach tol, the matrix is
 * refactored one precision up (fp8 -> bf16 -> fp32) and refinement goes on
 * from the current X.  max_iter bounds the refinement steps over all levels.
 */
int ir_solve(int n, int nrhs, const double *A, int lda, const double *B,
             int ldb, double *X, int ldx, const ir_opts *opts,
             ir_result *res, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solve requests on one GPU (no counterpart
 * in the paper; it is the request loop around the mixed-precision
 * factorization and refinement of ir_solve).
 * ------------------------------------------------------------------------- */
#define SERVE_PENDING   0
#define SERVE_RUNNING   1
#define SERVE_DONE      2
#define SERVE_FAILED    3
#define SERVE_FLAG_FAIL 1       /* dry-run only: the request reports failure */
#define SERVE_FLAG_BORROW 2     /* read A and B in place instead of copying them
                                   at enqueue; the caller keeps them unchanged
                                   until the ticket is retired by serve_poll   */

typedef struct serve_t serve_t;

typedef struct {
    size_t hbm_budget_bytes;    /* device memory the server may use            */
    int max_slots;              /* requests in flight at once (default 4)      */
    int precision;              /* default factorization precision (BF16)      */
    double tol;                 /* default backward-error target (1e-12)       */
    int max_queue;              /* pending requests allowed per path (slots,
                                   shared batches; 0: unlimited)                */
    int dry_run;                /* 1: scheduler test mode, no device work: each
                                   request holds its budget for a time
                                   proportional to n^3 and computes nothing    */
    int batch_n_max;            /* requests with n up to this share batched
                                   launches (binary32 factors, binary64
                                   refinement); 0: 1024, -1: none; <= 1024     */
    int batch_max;              /* most requests in one shared batch (0: 256)  */
    int reserved[2];            /* must be zero                                 */
} serve_cfg;

typedef struct {
    int n, nrhs;                /* 1 <= nrhs <= 64                              */
    const double *A;            /* n x n row-major, lda >= n                    */
    int lda;
    const double *B;            /* n x nrhs row-major, ldb >= nrhs              */
    int ldb;
    int device_inputs;          /* 0: A and B are host pointers; 1: device      */
    uint64_t matrix_id;         /* nonzero: cache the factors under this id; a
                                   later request with the same id and n must
                                   carry the same A and reuses them            */
    double tol;                 /* 0: the server default                        */
    int precision;              /* 0: the server default                        */
    int flags;                  /* SERVE_FLAG_*                                  */
    int reserved[4];
} serve_req;

typedef struct {
    int status;                 /* SERVE_*                                       */
    int error;                  /* LU_E* when failed                             */
    double eta;                 /* final backward error                          */
    double latency_s;           /* enqueue -> done                               */
    double queue_s;             /* enqueue -> start                              */
    int iters, gmres_iters, path, precision;   /* as ir_result                  */
    int cache_hit;              /* factors came from the cache                   */
    int batched;                /* solved in a shared batched launch             */
} serve_status;

typedef struct {
    size_t budget_bytes, used_bytes, peak_bytes;
    int queued, running, peak_running;
    long long completed, failed, cache_hits, evictions;
    int cache_entries;
    long long batches;          /* shared batched launches run                   */
    long long batched;          /* requests solved in them                       */
} serve_stats;

/* Create a server (its worker threads and streams) on the current device.
 * Returns 0, -1 for a bad cfg, -2 for a null handle pointer. */
int serve_create(const serve_cfg *cfg, serve_t **h);
/* Copy a request and queue it.  Returns 0 with *ticket set, -2 for bad
 * request fields, LU_EBUSY when it can never fit the budget, the queue is
 * full or the server is stopping.  The caller may free A and B on return,
 * unless the request carries SERVE_FLAG_BORROW. */
int serve_enqueue(serve_t *h, const serve_req *r, uint64_t *ticket);
/* Non-blocking.  Fills st; once st->status is SERVE_DONE the solution is
 * copied to X (host, n x nrhs row-major, may be NULL) and the ticket is
 * retired (a later poll returns LU_ENOTFOUND); a failed request is retired
 * the same way. */
int serve_poll(serve_t *h, uint64_t ticket, serve_status *st, double *X);
int serve_get_stats(serve_t *h, serve_stats *out);
/* Stop the workers (pending requests fail, running ones finish), free the
 * factor cache.  */
int serve_destroy(serve_t *h);

/* ---------------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper's algorithm: they time it).
 * While a session is open, every kernel launch of the library is bracketed
 * by CUDA events recorded on the launch's stream; lu_prof_end waits for
 * those events and returns, per launch class, the launch count, the summed
 * event time and the summed algorithmic work (flops; bytes where a class is
 * memory-bound).  Process-wide, one session at a time, host thread-safe.
 * ------------------------------------------------------------------------- */
#define LU_PROF_TSLU      0   /* tournament levels (TournPivot)                 */
#define LU_PROF_PIVOT     1   /* pivot bookkeeping and row moves                */
#define LU_PROF_TRSM_L21  2   /* FactorizeA10                                    */
#define LU_PROF_TRSM_U12  3   /* FactorizeA01                                    */
#define LU_PROF_SCHUR     4   /* FactorizeA11, binary64                          */
#define LU_PROF_SCHUR_LP  5   /* FactorizeA11, bf16/fp8 tensor cores             */
#define LU_PROF_SOLVE     6   /* getrs kernels                                   */
#define LU_PROF_RESIDUAL  7   /* binary64 residual and backward error            */
#define LU_PROF_OTHER     8   /* conversions, copies, scaling                    */
#define LU_PROF_CHOL_DIAG 9   /* Cholesky diagonal-block factorization           */
#define LU_PROF_SYRK      10  /* Cholesky trailing update (lower triangle)       */
#define LU_PROF_MATVEC32  11  /* Krylov products with binary32 multiplies        */
#define LU_PROF_NCLASS    12

typedef struct {
    int kernel_class;        /* LU_PROF_*                                        */
    int launches;            /* launches recorded                                */
    double total_ms;         /* summed CUDA-event time of those launches         */
    double total_flops;      /* summed algorithmic flops                         */
    double total_bytes;      /* summed algorithmic bytes                         */
} lu_prof_entry;

/* Open a session (discarding any previous records).  Returns 0. */
int lu_prof_begin(void);
/* Close the session: synchronises the recorded events and writes up to
 * max_entries non-empty classes to out (host array), their number to
 * *n_entries (host).  Returns 0, -2/-3 on bad arguments, LU_ELAUNCH if an
 * event failed. */
int lu_prof_end(lu_prof_entry *out, int max_entries, int *n_entries);
/* Kernels launched by this library in this process so far. */
unsigned long long lu_kernel_launch_count(void);

/* ---------------------------------------------------------------------------
 * Bounded device waits (no counterpart in the paper).  The library's kernels
 * wait on each other's progress in two places: the tensor-core Schur update
 * (mbarrier waits between its copy, MMA and epilogue warps) and the
 * work-list triangular solve (a work item waits for the items it depends
 * on).  Each such wait gives up after a wall-clock deadline (default 4 s,
 * read on the device from %globaltimer); the kernel then stops taking work,
 * waits for its own copies and MMAs in flight, frees its tensor memory and
 * exits, and the call reports LU_ETIMEOUT (the factorizations through
 * *info = -LU_ETIMEOUT, the solves through their return value).
 * ------------------------------------------------------------------------- */
#define LU_WAIT_SITE_TC     0   /* tcgen05 Schur update (lu_gemm_lowp, the
                                   bf16 / fp8 factorization, ir_solve)          */
#define LU_WAIT_SITE_SOLVE  1   /* work-list triangular solves                  */
#define LU_WAIT_NSITES      2

/*
 * lu_test_wait_config -- TEST HOOK: set the dependency-wait deadline of one
 * wait site (wait_ns > 0; 0 restores the 4 s default) and, with inject = 1,
 * make every later launch at that site first wait once on something that is
 * never signalled (an mbarrier nothing arrives on; a counter nothing
 * increments), so that the wait runs out after wait_ns and the error path
 * runs without a device fault.  Process-wide; applies to launches made after
 * the call.  Returns 0, -1 bad site, -2 wait_ns < 0 or > 600 s, -3 inject
 * not 0 or 1.
 */
int lu_test_wait_config(int site, long long wait_ns, int inject);

/* The deadline in nanoseconds that launches at `site` use now, or -1 for a
 * bad site. */
long long lu_wait_deadline_ns(int site);

#ifdef __cplusplus
}
#endif

#endif /* CONFLUX_LU_H */
