/*
 * lu_oracle_body.h -- the oracle's factorization and solve, written once for
 * an element type REAL with its fused multiply-add FMA and absolute value
 * FABS; FN(name) gives the instance's function name.  Included by
 * lu_oracle.c for binary64 (the reference form) and binary32 (the check of
 * the all-fp32 GPU factorization).  TEST INFRASTRUCTURE ONLY.
 */
/* ------------------------------------------------------------------------ */
/* Local LUP candidate selection (Section 7.3).  rows[0..nr) are row          */
/* positions of A; the panel is columns [k, k+w).  sel receives min(nr, w)    */
/* row positions in pivot order.                                              */
/* ------------------------------------------------------------------------ */
static void FN(gepp_select)(const REAL *A, int lda, int k, int w,
                        const int *rows, int nr, int *sel)
{
    REAL *W = (REAL *)malloc((size_t)nr * (size_t)w * sizeof(REAL));
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
        REAL bv = FABS(W[(size_t)c * w + c]);
        for (int i = c + 1; i < nr; ++i) {
            REAL v = FABS(W[(size_t)i * w + c]);
            if (v > bv || (v == bv && id[i] < id[best])) {
                best = i;
                bv = v;
            }
        }
        if (best != c) {
            for (int j = 0; j < w; ++j) {
                REAL t = W[(size_t)c * w + j];
                W[(size_t)c * w + j] = W[(size_t)best * w + j];
                W[(size_t)best * w + j] = t;
            }
            int t = id[c];
            id[c] = id[best];
            id[best] = t;
        }
        REAL piv = W[(size_t)c * w + c];
        if (piv != 0) {
            for (int i = c + 1; i < nr; ++i) {
                REAL l = W[(size_t)i * w + c] / piv;
                W[(size_t)i * w + c] = l;
                for (int j = c + 1; j < w; ++j)
                    W[(size_t)i * w + j] = FMA(-l, W[(size_t)c * w + j], W[(size_t)i * w + j]);
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
int FN(oracle_tslu_select)(int m, int lda, const REAL *A, int k, int w, int h, int *win)
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
        FN(gepp_select)(A, lda, k, w, rows, nr, &cur[(size_t)f * cap]);
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
                FN(gepp_select)(A, lda, k, w, stack, ns, dst);
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
int FN(oracle_lu_factor_q)(int m, int n, REAL *A, int lda, int b, int h,
                     int *piv, int *info, oracle_counts *cnt, int lowp);

int FN(oracle_lu_factor)(int m, int n, REAL *A, int lda, int b, int h,
                     int *piv, int *info, oracle_counts *cnt)
{
    return FN(oracle_lu_factor_q)(m, n, A, lda, b, h, piv, info, cnt, 0);
}

/* lowp = 0: every update in REAL.  lowp = 1 (bf16) / 2 (fp8 e4m3): the Schur
 * update (step 6) uses the rounded operands of oracle_gemm_lowp, with one
 * scale block per 256 rows of L21 and per 256 columns of U12 counted from
 * the step's first trailing row / column, sums in binary64 and one rounding
 * of the result to REAL. */
int FN(oracle_lu_factor_q)(int m, int n, REAL *A, int lda, int b, int h,
                     int *piv, int *info, oracle_counts *cnt, int lowp)
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
        FN(oracle_tslu_select)(m, lda, A, k, w, h, win);

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
                REAL *ra = &IDX(A, lda, k + j, 0), *rb = &IDX(A, lda, p, 0);
                for (int c = 0; c < n; ++c) {
                    REAL t = ra[c];
                    ra[c] = rb[c];
                    rb[c] = t;
                }
            }
        }

        /* 3. A00: no-pivot LU of the w x w block */
        for (int j = 0; j < w; ++j) {
            REAL u = IDX(A, lda, k + j, k + j);
            if (u == 0 && *info == 0)
                *info = k + j + 1;
            for (int i = j + 1; i < w; ++i) {
                REAL l;
                if (u != 0) {
                    l = IDX(A, lda, k + i, k + j) / u;
                    ++c_div;
                } else {
                    l = 0;
                }
                IDX(A, lda, k + i, k + j) = l;
                for (int c = j + 1; c < w; ++c) {
                    IDX(A, lda, k + i, k + c) =
                        FMA(-l, IDX(A, lda, k + j, k + c), IDX(A, lda, k + i, k + c));
                    ++c_fma;
                }
            }
        }

        /* 4. L21 = A21 * U00^{-1}: column by column, forward */
        long long fma_l21 = 0, div_l21 = 0;
#pragma omp parallel for schedule(static) reduction(+ : fma_l21, div_l21)
        for (int i = k + w; i < m; ++i) {
            REAL *row = &IDX(A, lda, i, 0);
            for (int j = 0; j < w; ++j) {
                REAL a = row[k + j];
                for (int p = 0; p < j; ++p) {
                    a = FMA(-row[k + p], IDX(A, lda, k + p, k + j), a);
                    ++fma_l21;
                }
                REAL u = IDX(A, lda, k + j, k + j);
                if (u != 0) {
                    row[k + j] = a / u;
                    ++div_l21;
                } else {
                    row[k + j] = 0;
                }
            }
        }
        c_fma += fma_l21;
        c_div += div_l21;

        /* 5. U12 = L00^{-1} * A12: row by row, forward */
        for (int i = 1; i < w; ++i) {
            REAL *row = &IDX(A, lda, k + i, 0);
            for (int p = 0; p < i; ++p) {
                REAL l = row[k + p];
                const REAL *up = &IDX(A, lda, k + p, 0);
                for (int c = k + w; c < n; ++c) {
                    row[c] = FMA(-l, up[c], row[c]);
                    ++c_fma;
                }
            }
        }

        /* 6. A22 -= L21 * U12: for each element, p ascending */
        if (lowp && m - k - w > 0 && n - k - w > 0) {
            int M = m - k - w, N = n - k - w;
            float *Lf = (float *)malloc((size_t)M * w * sizeof(float));
            float *Uf = (float *)malloc((size_t)w * N * sizeof(float));
            float *Cf = (float *)malloc((size_t)M * N * sizeof(float));
            double *Cr = (double *)malloc((size_t)M * N * sizeof(double));
            double *Sa = (double *)malloc((size_t)M * N * sizeof(double));
            for (int i = 0; i < M; ++i)
                for (int p = 0; p < w; ++p)
                    Lf[(size_t)i * w + p] = (float)IDX(A, lda, k + w + i, k + p);
            for (int p = 0; p < w; ++p)
                for (int j = 0; j < N; ++j)
                    Uf[(size_t)p * N + j] = (float)IDX(A, lda, k + p, k + w + j);
            for (int i = 0; i < M; ++i)
                for (int j = 0; j < N; ++j)
                    Cf[(size_t)i * N + j] = (float)IDX(A, lda, k + w + i, k + w + j);
            oracle_gemm_lowp(M, N, w, Lf, w, Uf, N, Cf, N, lowp == 2, Cr, Sa);
            for (int i = 0; i < M; ++i)
                for (int j = 0; j < N; ++j)
                    IDX(A, lda, k + w + i, k + w + j) = (REAL)Cr[(size_t)i * N + j];
            free(Lf);
            free(Uf);
            free(Cf);
            free(Cr);
            free(Sa);
            continue;
        }
        long long fma_s = 0;
#pragma omp parallel for schedule(static) reduction(+ : fma_s)
        for (int i = k + w; i < m; ++i) {
            REAL *row = &IDX(A, lda, i, 0);
            for (int p = 0; p < w; ++p) {
                REAL l = row[k + p];
                const REAL *up = &IDX(A, lda, k + p, 0);
                for (int c = k + w; c < n; ++c)
                    row[c] = FMA(-l, up[c], row[c]);
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
int FN(oracle_lu_solve)(int n, int nrhs, const REAL *LU, int lda, const int *piv,
                    REAL *B, int ldb)
{
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -7;
    for (int i = 0; i < n; ++i) {
        int p = piv[i];
        if (p != i)
            for (int c = 0; c < nrhs; ++c) {
                REAL t = IDX(B, ldb, i, c);
                IDX(B, ldb, i, c) = IDX(B, ldb, p, c);
                IDX(B, ldb, p, c) = t;
            }
    }
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < i; ++p) {
            REAL l = IDX(LU, lda, i, p);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = FMA(-l, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
    for (int i = n - 1; i >= 0; --i) {
        for (int p = i + 1; p < n; ++p) {
            REAL u = IDX(LU, lda, i, p);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = FMA(-u, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
        REAL d = IDX(LU, lda, i, i);
        for (int c = 0; c < nrhs; ++c)
            IDX(B, ldb, i, c) = IDX(B, ldb, i, c) / d;
    }
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Cholesky factorization A = L L^T of a symmetric positive definite n x n   */
/* matrix (Section 2.2 names Cholesky as a further kernel for the same       */
/* schedule; the Conclusions name it as the next one).  Right-looking, one   */
/* column at a time, reading and writing the lower triangle only:            */
/*   l_jj = sqrt(a_jj);  l_ij = a_ij / l_jj (i > j);                          */
/*   a_ic = fma(-l_ij, l_cj, a_ic) for j < c <= i,                             */
/* so every element receives its update terms in ascending j before its     */
/* own square root or division.  The first column whose a_jj is not > 0     */
/* (or is NaN) stops the factorization with *info = j + 1 (LAPACK potrf's   */
/* convention); columns before it hold L, the rest is as far as it got.     */
/* The strict upper triangle is not referenced.                              */
/* ------------------------------------------------------------------------ */
int FN(oracle_chol_factor)(int n, REAL *A, int lda, int *info)
{
    if (n < 0) return -1;
    if (lda < (n > 1 ? n : 1)) return -3;
    *info = 0;
    for (int j = 0; j < n; ++j) {
        REAL d = IDX(A, lda, j, j);
        if (!(d > (REAL)0)) {
            *info = j + 1;
            return 0;
        }
        REAL ljj = SQRT(d);
        IDX(A, lda, j, j) = ljj;
        for (int i = j + 1; i < n; ++i)
            IDX(A, lda, i, j) = IDX(A, lda, i, j) / ljj;
        for (int i = j + 1; i < n; ++i) {
            REAL lij = IDX(A, lda, i, j);
            for (int c = j + 1; c <= i; ++c)
                IDX(A, lda, i, c) = FMA(-lij, IDX(A, lda, c, j), IDX(A, lda, i, c));
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Solve A X = B with the Cholesky factor L (lower triangle of L):           */
/* L Y = B by forward substitution, then L^T X = Y by backward              */
/* substitution; each element receives its terms in ascending (forward) or */
/* descending (backward) index order and then one division by l_ii.         */
/* B is n x nrhs row-major (ldb >= nrhs), overwritten with X.               */
/* ------------------------------------------------------------------------ */
int FN(oracle_chol_solve)(int n, int nrhs, const REAL *L, int lda, REAL *B, int ldb)
{
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (ldb < (nrhs > 1 ? nrhs : 1)) return -6;
    for (int i = 0; i < n; ++i) {
        for (int p = 0; p < i; ++p) {
            REAL l = IDX(L, lda, i, p);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = FMA(-l, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
        REAL d = IDX(L, lda, i, i);
        for (int c = 0; c < nrhs; ++c)
            IDX(B, ldb, i, c) = IDX(B, ldb, i, c) / d;
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int p = n - 1; p > i; --p) {
            REAL l = IDX(L, lda, p, i);
            for (int c = 0; c < nrhs; ++c)
                IDX(B, ldb, i, c) = FMA(-l, IDX(B, ldb, p, c), IDX(B, ldb, i, c));
        }
        REAL d = IDX(L, lda, i, i);
        for (int c = 0; c < nrhs; ++c)
            IDX(B, ldb, i, c) = IDX(B, ldb, i, c) / d;
    }
    return 0;
}
