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

/* ------------------------------------------------------------------------ */
/* Local LUP candidate selection (Section 7.3).  rows[0..nr) are row          */
/* positions of A; the panel is columns [k, k+w).  sel receives min(nr, w)    */
/* row positions in pivot order.                                              */
/* ------------------------------------------------------------------------ */
static void gepp_select(const double *A, int lda, int k, int w,
                        const int *rows, int nr, int *sel)
{
    double *W = (double *)malloc((size_t)nr * (size_t)w * sizeof(double));
    int *id = (int *)malloc((size_t)nr * sizeof(int));
    for (int i = 0; i < nr; ++i) {
        id[i] = rows[i];
        for (int j = 0; j < w; ++j)
            W[(size_t)i * w + j] = IDX(A, lda, rows[i], k + j);
    }
    int ns = nr < w ? nr : w;
    for (int c = 0; c < ns; ++c) {
        /* argmax |W[i][c]| over i >= c; a tie goes to the smallest position */
        int best = c;
        double bv = fabs(W[(size_t)c * w + c]);
        for (int i = c + 1; i < nr; ++i) {
            double v = fabs(W[(size_t)i * w + c]);
            if (v > bv || (v == bv && id[i] < id[best])) {
                best = i;
                bv = v;
            }
        }
        if (best != c) {
            for (int j = 0; j < w; ++j) {
                double t = W[(size_t)c * w + j];
                W[(size_t)c * w + j] = W[(size_t)best * w + j];
                W[(size_t)best * w + j] = t;
            }
            int t = id[c];
            id[c] = id[best];
            id[best] = t;
        }
        double piv = W[(size_t)c * w + c];
        if (piv != 0.0) {
            for (int i = c + 1; i < nr; ++i) {
                double l = W[(size_t)i * w + c] / piv;
                W[(size_t)i * w + c] = l;
                for (int j = c + 1; j < w; ++j)
                    W[(size_t)i * w + j] = fma(-l, W[(size_t)c * w + j], W[(size_t)i * w + j]);
            }
        }
    }
    for (int i = 0; i < ns; ++i)
        sel[i] = id[i];
    free(W);
    free(id);
}

/* ------------------------------------------------------------------------ */
/* TournPivot over active rows [k, m) and panel columns [k, k+w) (Section     */
/* 7.3).  win receives w row positions (w <= m-k) in the root's pivot order.  */
/* Returns 0, or -1 on bad arguments.                                         */
/* ------------------------------------------------------------------------ */
int oracle_tslu_select(int m, int lda, const double *A, int k, int w, int h, int *win)
{
    int nact = m - k;
    if (w <= 0 || h <= 0 || nact < w)
        return -1;
    int nleaf = (nact + h - 1) / h;
    int cap = (h > 2 * w ? h : 2 * w);
    int *cur = (int *)malloc((size_t)nleaf * cap * sizeof(int));
    int *nxt = (int *)malloc((size_t)nleaf * cap * sizeof(int));
    int *ncur = (int *)malloc((size_t)nleaf * sizeof(int));
    int *nnxt = (int *)malloc((size_t)nleaf * sizeof(int));

    /* leaves: local LUP on h consecutive rows */
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < nleaf; ++f) {
        int r0 = k + f * h;
        int nr = (r0 + h <= m) ? h : (m - r0);
        int *rows = (int *)malloc((size_t)nr * sizeof(int));
        for (int i = 0; i < nr; ++i)
            rows[i] = r0 + i;
        gepp_select(A, lda, k, w, rows, nr, &cur[(size_t)f * cap]);
        ncur[f] = nr < w ? nr : w;
        free(rows);
    }
    /* playoff rounds: pair (0,1), (2,3), ...; an odd last node goes up */
    int nnode = nleaf;
    while (nnode > 1) {
        int npar = (nnode + 1) / 2;
#pragma omp parallel for schedule(dynamic)
        for (int p = 0; p < npar; ++p) {
            int l = 2 * p, r = 2 * p + 1;
            int *dst = &nxt[(size_t)p * cap];
            if (r >= nnode) {
                memcpy(dst, &cur[(size_t)l * cap], (size_t)ncur[l] * sizeof(int));
                nnxt[p] = ncur[l];
            } else {
                int ns = ncur[l] + ncur[r];
                int *stack = (int *)malloc((size_t)ns * sizeof(int));
                memcpy(stack, &cur[(size_t)l * cap], (size_t)ncur[l] * sizeof(int));
                memcpy(stack + ncur[l], &cur[(size_t)r * cap], (size_t)ncur[r] * sizeof(int));
                gepp_select(A, lda, k, w, stack, ns, dst);
                nnxt[p] = ns < w ? ns : w;
                free(stack);
            }
        }
        int *t = cur; cur = nxt; nxt = t;
        int *tn = ncur; ncur = nnxt; nnxt = tn;
        nnode = npar;
    }
    /* A single leaf is its own root: its selection is already in pivot order. */
    memcpy(win, cur, (size_t)w * sizeof(int));
    free(cur);
    free(nxt);
    free(ncur);
    free(nnxt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Blocked right-looking LU with tournament pivoting (Algorithm 1 on one      */
/* node).  A is m x n row-major (lda >= n).  piv has min(m,n) entries:        */
/* piv[i] = the 0-based row swapped with row i at step i (LAPACK ipiv,        */
/* 0-based).  info = 0, or j+1 for the first j with U(j,j) == 0.              */
/* cnt may be NULL.  nthreads > 1 parallelises independent row loops only;   */
/* each element's operation sequence is the same for every thread count.    */
/* Returns 0, or a negative argument index on bad arguments.                  */
/* ------------------------------------------------------------------------ */
int oracle_lu_factor(int m, int n, double *A, int lda, int b, int h,
                     int *piv, int *info, oracle_counts *cnt)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (b < 1) return -5;
    if (h < 1) return -6;
    int kmax = m < n ? m : n;
    long long c_div = 0, c_fma = 0;
    *info = 0;
    int *win = (int *)malloc((size_t)(b > 0 ? b : 1) * sizeof(int));
    for (int k = 0; k < kmax; k += b) {
        int w = (kmax - k) < b ? (kmax - k) : b;

        /* 1. TournPivot on the current values of the panel */
        oracle_tslu_select(m, lda, A, k, w, h, win);

        /* 2. sequential swaps: winner j goes to row k+j; track where the
         *    rows of the top block move so later winners are found */
        for (int j = 0; j < w; ++j) {
            int p = win[j];
            /* a winner that sat in a top row already moved may have moved */
            for (int jj = 0; jj < j; ++jj)
                if (p == k + jj)
                    p = piv[k + jj];
            piv[k + j] = p;
            if (p != k + j) {
                double *ra = &IDX(A, lda, k + j, 0), *rb = &IDX(A, lda, p, 0);
                for (int c = 0; c < n; ++c) {
                    double t = ra[c];
                    ra[c] = rb[c];
                    rb[c] = t;
                }
            }
        }

        /* 3. A00: no-pivot LU of the w x w block */
        for (int j = 0; j < w; ++j) {
            double u = IDX(A, lda, k + j, k + j);
            if (u == 0.0 && *info == 0)
                *info = k + j + 1;
            for (int i = j + 1; i < w; ++i) {
                double l;
                if (u != 0.0) {
                    l = IDX(A, lda, k + i, k + j) / u;
                    ++c_div;
                } else {
                    l = 0.0;
                }
                IDX(A, lda, k + i, k + j) = l;
                for (int c = j + 1; c < w; ++c) {
                    IDX(A, lda, k + i, k + c) =
                        fma(-l, IDX(A, lda, k + j, k + c), IDX(A, lda, k + i, k + c));
                    ++c_fma;
                }
            }
        }

        /* 4. L21 = A21 * U00^{-1}: column by column, forward */
        long long fma_l21 = 0, div_l21 = 0;
#pragma omp parallel for schedule(static) reduction(+ : fma_l21, div_l21)
        for (int i = k + w; i < m; ++i) {
            double *row = &IDX(A, lda, i, 0);
            for (int j = 0; j < w; ++j) {
                double a = row[k + j];
                for (int p = 0; p < j; ++p) {
                    a = fma(-row[k + p], IDX(A, lda, k + p, k + j), a);
                    ++fma_l21;
                }
                double u = IDX(A, lda, k + j, k + j);
                if (u != 0.0) {
                    row[k + j] = a / u;
                    ++div_l21;
                } else {
                    row[k + j] = 0.0;
                }
            }
        }
        c_fma += fma_l21;
        c_div += div_l21;

        /* 5. U12 = L00^{-1} * A12: row by row, forward */
        for (int i = 1; i < w; ++i) {
            double *row = &IDX(A, lda, k + i, 0);
            for (int p = 0; p < i; ++p) {
                double l = row[k + p];
                const double *up = &IDX(A, lda, k + p, 0);
                for (int c = k + w; c < n; ++c) {
                    row[c] = fma(-l, up[c], row[c]);
                    ++c_fma;
                }
            }
        }

        /* 6. A22 -= L21 * U12: for each element, p ascending */
        long long fma_s = 0;
#pragma omp parallel for schedule(static) reduction(+ : fma_s)
        for (int i = k + w; i < m; ++i) {
            double *row = &IDX(A, lda, i, 0);
            for (int p = 0; p < w; ++p) {
                double l = row[k + p];
                const double *up = &IDX(A, lda, k + p, 0);
                for (int c = k + w; c < n; ++c)
                    row[c] = fma(-l, up[c], row[c]);
                fma_s += (n - k - w) > 0 ? (n - k - w) : 0;
            }
        }
        c_fma += fma_s;
    }
    free(win);
    if (cnt) {
        cnt->s1_div = c_div;
        cnt->s2_fma = c_fma;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Solve A X = B with the factors of oracle_lu_factor (n x n):               */
/* X = U^{-1} L^{-1} P B.  B is n x nrhs row-major (ldb >= nrhs), overwritten.*/
/* ------------------------------------------------------------------------ */
int oracle_lu_solve(int n, int nrhs, const double *LU, int lda, const int *piv,
                    double *B, int ldb)
{
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -7;
    for (int i = 0; i < n; ++i) {
        int p = piv[i];
        if (p != i)
            for (int c = 0; c < nrhs; ++c) {
                double t = IDX(B, ldb, i, c);
                IDX(B, ldb, i, c) = IDX(B, ldb, p, c);
                IDX(B, ldb, p, c) = t;
            }
    }
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < i; ++p) {
            double l = IDX(LU, lda, i, p);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = fma(-l, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
    for (int i = n - 1; i >= 0; --i) {
        for (int p = i + 1; p < n; ++p) {
            double u = IDX(LU, lda, i, p);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = fma(-u, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
        double d = IDX(LU, lda, i, i);
        for (int c = 0; c < nrhs; ++c)
            IDX(B, ldb, i, c) = IDX(B, ldb, i, c) / d;
    }
    return 0;
}

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
