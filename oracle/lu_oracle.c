/*
 * lu_oracle.c -- the CPU oracle for the tournament-pivoting LU hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library shares
 * no code, header, table or helper with it, and neither includes the other.
 *
 * What it computes (plain, slow, FP64, IEEE-754 binary64 round-to-nearest,
 * true division, one fused multiply-add per update term):
 *
 *   In-place LU, PA = LU, of a row-major m x n matrix, right-looking and
 *   blocked by v = b columns (the COnfLUX outer loop of Algorithm 1 and the
 *   "Computation Routines" of Section 7.2).  Each step k:
 *     1. TournPivot (Section 7.3 "Pivoting in COnfLUX" and the step-1 text of
 *        the I/O-cost proof in Section 7.4): the active rows are cut into
 *        leaves of h consecutive rows; each leaf runs a local LUP (GEPP) on
 *        its panel rows and keeps v candidate rows; candidates meet in
 *        ceil(log2) rounds of a pairwise "playoff" (adjacent nodes, lower
 *        first, an odd last node goes up unchanged); each meeting is a GEPP
 *        on the current panel values of the stacked candidates.  The root's
 *        candidates, in its pivot order, are the v pivot rows; the root also
 *        yields the factored A00.
 *     2. The pivot rows are brought to the top of the active block with
 *        LAPACK-style sequential row swaps over all n columns (the swap
 *        order fixes the row positions that the next step's leaves use; a
 *        row mask with the same logical order gives the same factors).
 *     3. A00: no-pivot LU of the v x v block (statement S1 A[i,k] /= A[k,k],
 *        statement S2 A[i,j] -= A[i,k]*A[k,j]; Fig. 1 and Section 6).
 *     4. FactorizeA10: L21 = A21 * U00^{-1}   (triangular solve, Section 7.2)
 *     5. FactorizeA01: U12 = L00^{-1} * A12   (unit lower, Section 7.2)
 *     6. FactorizeA11: A22 -= L21 * U12        (Schur update, Section 7.2)
 *
 * Readings where the paper is silent:
 *   - leaves are h consecutive active rows (the paper gives each processor a
 *     contiguous share of the rows);
 *   - a tie in |value| goes to the smallest row position;
 *   - upper tree levels compare the candidates' CURRENT panel values (the
 *     CALU reading of "exchange v x v blocks");
 *   - a column whose pivot is exactly zero is skipped in the GEPP selection
 *     (no division); in A00 and L21 such a column of L is set to zero and
 *     info records the first one (1-based), as LAPACK getrf does.
 *
 * The same file holds the Cholesky factorization A = L L^T and its solve
 * (the kernel Section 2.2 and the Conclusions name for the same schedule;
 * no pivoting): right-looking, lower triangle only, one fused multiply-add
 * per update term, then the column's square root or division.
 *
 * Every update term is a = fma(-l, u, a) with the summation index ascending,
 * so any blocking that keeps that per-element order gives bit-identical
 * numbers.  Build with -ffp-contract=off so that no other expression fuses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(A, lda, i, j) ((A)[(size_t)(i) * (size_t)(lda) + (size_t)(j)])

/* Counters for the loop-bound pins of Section 6: S1 divisions and S2 fused
 * updates performed on the matrix itself (tournament copies excluded). */
typedef struct {
    long long s1_div;
    long long s2_fma;
} oracle_counts;

void oracle_gemm_lowp(int M, int N, int K, const float *L, int ldl, const float *U, int ldu,
                      const float *C, int ldc, int fp8, double *Cref, double *Sabs);

#define REAL double
#define FMA fma
#define FABS fabs
#define SQRT sqrt
#define FN(name) name
#include "lu_oracle_body.h"
#undef REAL
#undef FMA
#undef FABS
#undef SQRT
#undef FN

#define REAL float
#define FMA fmaf
#define FABS fabsf
#define SQRT sqrtf
#define FN(name) name##_f32
#include "lu_oracle_body.h"
#undef REAL
#undef FMA
#undef FABS
#undef SQRT
#undef FN

/* ------------------------------------------------------------------------ */
/* Relative backward error per right-hand side (FP64):                       */
/*   eta_c = ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf).     */
/* The paper does not define a stopping test; this is the normwise           */
/* backward error of Rigal and Gaches.  eta has nrhs entries.                 */
/* ------------------------------------------------------------------------ */
void oracle_backward_error(int n, int nrhs, const double *A, int lda,
                           const double *B, int ldb, const double *X, int ldx,
                           double *eta)
{
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            s += fabs(IDX(A, lda, i, j));
        if (s > anorm)
            anorm = s;
    }
    for (int c = 0; c < nrhs; ++c) {
        double rmax = 0.0, xmax = 0.0, bmax = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = IDX(B, ldb, i, c);
            for (int j = 0; j < n; ++j)
                r = fma(-IDX(A, lda, i, j), IDX(X, ldx, j, c), r);
            if (fabs(r) > rmax) rmax = fabs(r);
            if (fabs(IDX(X, ldx, i, c)) > xmax) xmax = fabs(IDX(X, ldx, i, c));
            if (fabs(IDX(B, ldb, i, c)) > bmax) bmax = fabs(IDX(B, ldb, i, c));
        }
        double den = anorm * xmax + bmax;
        eta[c] = den > 0.0 ? rmax / den : 0.0;
    }
}

/* Thread count for the row-parallel loops (timing only; results do not
 * depend on it).  Returns the count in effect. */
#ifdef _OPENMP
#include <omp.h>
#endif
int oracle_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Low-precision operands of the mixed-precision Schur update (the paper is */
/* silent on precision).  Written from the format definitions:              */
/*   bfloat16: the upper 16 bits of binary32, round to nearest, ties even.  */
/*   fp8 e4m3 (OCP): 4 exponent bits (bias 7), 3 fraction bits, subnormal   */
/*   spacing 2^-9, largest finite 448; round to nearest, ties even, and     */
/*   saturate to +-448.                                                      */
/* ------------------------------------------------------------------------ */
float oracle_round_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u)
        return x;
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

float oracle_round_e4m3(float x)
{
    if (x != x)
        return x;
    double a = fabs((double)x);
    if (a == 0.0)
        return x;
    int e;
    frexp(a, &e);            /* a in [2^(e-1), 2^e) */
    int k = e - 1;
    if (k < -6)
        k = -6;              /* subnormal range: fixed spacing 2^-9 */
    double q = ldexp(1.0, k - 3);
    double r = rint(a / q) * q;
    if (r > 448.0)
        r = 448.0;
    return (float)(x < 0 ? -r : r);
}

/* Smallest e with maxabs * 2^-e <= 448, decided in binary32 (v = maxabs/448
 * rounded to float), the precision the GPU decides it in. */
int oracle_e4m3_exponent(float maxabs)
{
    if (!(maxabs > 0.0f) || isinf(maxabs))
        return 0;
    float v = maxabs / 448.0f;
    int e;
    float f = frexpf(v, &e);
    return (f == 0.5f) ? e - 1 : e;
}

/* Reference of the scaled low-precision update, one 256 x 256 scale tile per
 * operand block:
 *   Cref[i][j] = C[i][j] - 2^(eL(i/256) + eU(j/256)) * sum_p qL[i][p] qU[p][j]
 * with qL = round(L * 2^-eL), qU = round(U * 2^-eU), sums in binary64, and
 * Sabs[i][j] = 2^(eL+eU) * sum_p |qL qU| (for error bounds).  fp8 = 0: bf16
 * operands, e = 0. */
void oracle_gemm_lowp(int M, int N, int K, const float *L, int ldl, const float *U, int ldu,
                      const float *C, int ldc, int fp8, double *Cref, double *Sabs)
{
    int nbm = (M + 255) / 256, nbn = (N + 255) / 256;
    int *eL = (int *)calloc((size_t)nbm + 1, sizeof(int));
    int *eU = (int *)calloc((size_t)nbn + 1, sizeof(int));
    if (fp8) {
        for (int b = 0; b < nbm; ++b) {
            float mx = 0.0f;
            for (int i = b * 256; i < M && i < b * 256 + 256; ++i)
                for (int p = 0; p < K; ++p)
                    if (fabsf(L[(size_t)i * ldl + p]) > mx)
                        mx = fabsf(L[(size_t)i * ldl + p]);
            eL[b] = oracle_e4m3_exponent(mx);
        }
        for (int b = 0; b < nbn; ++b) {
            float mx = 0.0f;
            for (int p = 0; p < K; ++p)
                for (int j = b * 256; j < N && j < b * 256 + 256; ++j)
                    if (fabsf(U[(size_t)p * ldu + j]) > mx)
                        mx = fabsf(U[(size_t)p * ldu + j]);
            eU[b] = oracle_e4m3_exponent(mx);
        }
    }
    double *qL = (double *)malloc((size_t)M * (K > 0 ? K : 1) * sizeof(double));
    double *qU = (double *)malloc((size_t)(K > 0 ? K : 1) * N * sizeof(double));
    for (int i = 0; i < M; ++i)
        for (int p = 0; p < K; ++p) {
            float x = ldexpf(L[(size_t)i * ldl + p], -eL[i / 256]);
            qL[(size_t)i * K + p] = fp8 ? oracle_round_e4m3(x) : oracle_round_bf16(x);
        }
    for (int p = 0; p < K; ++p)
        for (int j = 0; j < N; ++j) {
            float x = ldexpf(U[(size_t)p * ldu + j], -eU[j / 256]);
            qU[(size_t)p * N + j] = fp8 ? oracle_round_e4m3(x) : oracle_round_bf16(x);
        }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) {
            double s = 0.0, sa = 0.0;
            for (int p = 0; p < K; ++p) {
                double t = qL[(size_t)i * K + p] * qU[(size_t)p * N + j];
                s += t;
                sa += fabs(t);
            }
            int e = eL[i / 256] + eU[j / 256];
            Cref[(size_t)i * N + j] = (double)C[(size_t)i * ldc + j] - ldexp(s, e);
            Sabs[(size_t)i * N + j] = ldexp(sa, e);
        }
    free(qL);
    free(qU);
    free(eL);
    free(eU);
}

/* Elementwise roundings of an array (test access to the two quantizers). */
void oracle_round_array(const float *x, float *y, long long n, int fp8)
{
    for (long long i = 0; i < n; ++i)
        y[i] = fp8 ? oracle_round_e4m3(x[i]) : oracle_round_bf16(x[i]);
}
