"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test names what it pins.  None of them compares the oracle with itself:
they use LAPACK getrf (partial pivoting is the b = 1 and the one-leaf special
case of tournament pivoting), closed-form factors, exact integer determinants,
exact rational arithmetic and the vertex counts of Section 6.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from tests.exact_tournament import lu as exact_lu

EPS = 2.0 ** -53


def split_lu(LU):
    m, n = LU.shape
    k = min(m, n)
    L = np.tril(LU[:, :k], -1) + np.eye(m, k)
    U = np.triu(LU[:k, :])
    return L, U


def apply_piv(A, piv):
    PA = np.array(A, copy=True)
    for i, p in enumerate(piv):
        if p != i:
            PA[[i, p]] = PA[[p, i]]
    return PA


# --- special cases that reduce to partial pivoting (LAPACK getrf) ----------

@pytest.mark.parametrize("n,h", [(37, 4), (64, 16), (100, 128), (129, 7)])
def test_b1_equals_partial_pivoting(oracle_mod, n, h):
    """b = 1: every leaf keeps its largest |entry| and the playoff keeps the
    largest of those, so the pivots are LAPACK's (first maximum = smallest
    row, the same tie rule)."""
    A = wl.matrix_uniform(n, n, seed=10 + n)
    LU, piv, info = oracle_mod.lu_factor(A, b=1, h=h)
    lu_ref, ipiv = sla.lu_factor(A)
    assert info == 0
    np.testing.assert_array_equal(piv, ipiv)
    np.testing.assert_allclose(LU, lu_ref, rtol=0, atol=1e-12 * np.abs(lu_ref).max())


@pytest.mark.parametrize("n,b", [(50, 8), (96, 32), (131, 16), (200, 64)])
def test_single_leaf_equals_partial_pivoting(oracle_mod, n, b):
    """h >= number of rows: one leaf, whose local LUP is the root; the panel
    pivots are GEPP's and the block update reproduces getrf."""
    A = wl.matrix_normal(n, n, seed=20 + n)
    LU, piv, info = oracle_mod.lu_factor(A, b=b, h=n)
    lu_ref, ipiv = sla.lu_factor(A)
    assert info == 0
    np.testing.assert_array_equal(piv, ipiv)
    np.testing.assert_allclose(LU, lu_ref, rtol=0, atol=1e-11 * np.abs(lu_ref).max())


def test_tournament_differs_from_gepp_somewhere(oracle_mod):
    """A multi-leaf tree is a different rule from GEPP: on a seeded matrix it
    must pick at least one different pivot (guards against an oracle that
    silently ignores h)."""
    A = wl.matrix_uniform(256, 256, seed=3)
    _, piv_t, _ = oracle_mod.lu_factor(A, b=32, h=8)
    _, ipiv = sla.lu_factor(A)
    assert (piv_t != ipiv).any()


# --- closed forms ---------------------------------------------------------

@pytest.mark.parametrize("n,b,h", [(64, 8, 4), (100, 16, 8), (150, 32, 16), (77, 5, 3)])
def test_closed_form_lu_product(oracle_mod, n, b, h):
    """A = L U with |l_ij| <= 1/2 and |u_jj| >= 1: every row subset's Schur
    complement column is L[:,c] u_cc, so the diagonal row wins strictly at
    every tree node; piv = identity and the factors are L and U.  Entries are
    multiples of 1/16, so A and every Schur complement are exact in binary64
    and the factors must come back bit for bit."""
    ul = wl.uniform01(5, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    uu = wl.uniform01(6, n, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    L = np.tril(np.floor(ul * 17 - 8.5 + 0.5) / 16.0, -1) + np.eye(n)      # [-1/2, 1/2]
    U = np.triu(np.floor(uu * 33 - 16.5 + 0.5) / 16.0, 1)                  # [-1, 1]
    d = np.floor(np.diag(uu) * 17) / 16.0 + 1.0                            # [1, 2]
    U += np.diag(np.where(np.arange(n) % 2 == 0, d, -d))
    A = L @ U
    LU, piv, info = oracle_mod.lu_factor(A, b=b, h=h)
    assert info == 0
    np.testing.assert_array_equal(piv, np.arange(n))
    Lo, Uo = split_lu(LU)
    np.testing.assert_array_equal(Lo, L)
    np.testing.assert_array_equal(Uo, U)


@pytest.mark.parametrize("n,b,h", [(16, 4, 2), (33, 8, 3), (64, 16, 16), (40, 1, 5)])
def test_permutation_matrix(oracle_mod, n, b, h):
    """A = Q (a permutation): each panel column has one nonzero, zero ties
    elsewhere go to the smallest row; L = U = I exactly and the swaps
    reconstruct Q."""
    perm = np.argsort(wl.uniform01(9, n, np.arange(n, dtype=np.uint64)))
    Q = np.zeros((n, n))
    Q[np.arange(n), perm] = 1.0
    LU, piv, info = oracle_mod.lu_factor(Q, b=b, h=h)
    assert info == 0
    np.testing.assert_array_equal(LU, np.eye(n))
    np.testing.assert_array_equal(apply_piv(Q, piv), np.eye(n))


@pytest.mark.parametrize("n,b,h", [(20, 4, 2), (50, 8, 8), (31, 32, 4)])
def test_upper_triangular(oracle_mod, n, b, h):
    """Upper-triangular A with nonzero diagonal: only the diagonal row has a
    nonzero in its column, so P = I, L = I and U = A exactly."""
    U = np.triu(wl.matrix_uniform(n, n, seed=12))
    U[np.arange(n), np.arange(n)] += np.sign(U.diagonal()) * 0.5
    LU, piv, info = oracle_mod.lu_factor(U, b=b, h=h)
    assert info == 0
    np.testing.assert_array_equal(piv, np.arange(n))
    np.testing.assert_array_equal(LU, U)


def _det_exact(M):
    """Exact determinant by Laplace expansion along the first row (ints)."""
    n = len(M)
    if n == 1:
        return M[0][0]
    tot = 0
    for j in range(n):
        if M[0][j] == 0:
            continue
        minor = [row[:j] + row[j + 1:] for row in M[1:]]
        tot += (-1) ** j * M[0][j] * _det_exact(minor)
    return tot


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_cofactor_determinant(oracle_mod, n):
    """sign(piv) * prod(U_jj) equals the exact cofactor determinant of small
    integer matrices with entries in [-4, 4]."""
    for trial in range(6):
        u = wl.uniform01(100 + n, trial, np.arange(n * n, dtype=np.uint64))
        M = (np.floor(u * 9) - 4).astype(np.int64).reshape(n, n)
        exact = _det_exact(M.tolist())
        for b, h in [(1, 1), (2, 2), (3, 1), (n, 2)]:
            LU, piv, info = oracle_mod.lu_factor(M.astype(np.float64), b=b, h=h)
            sign = (-1) ** int(np.sum(piv != np.arange(n)))
            det = sign * np.prod(np.diag(LU))
            if exact == 0:
                assert info > 0 or abs(det) <= 1e-9 * 4.0 ** n
            else:
                assert abs(det - exact) <= 1e-13 * abs(exact) * 10, (M, b, h, det, exact)


def test_singular_column_sets_info(oracle_mod):
    """A zero column gives an exact zero pivot: info = its index + 1, the L
    column is zero, no NaN is produced (reading of getrf's convention)."""
    n = 12
    A = wl.matrix_uniform(n, n, seed=4)
    A[:, 5] = 0.0
    LU, piv, info = oracle_mod.lu_factor(A, b=4, h=3)
    assert info == 6
    assert np.isfinite(LU).all()
    np.testing.assert_array_equal(LU[6:, 5], 0.0)


# --- invariants -----------------------------------------------------------

@pytest.mark.parametrize("m,n,b,h", [(128, 128, 32, 16), (300, 300, 64, 128), (257, 257, 32, 128),
                                     (200, 120, 16, 8), (120, 200, 16, 8), (512, 512, 32, 128)])
def test_backward_stability_invariants(oracle_mod, m, n, b, h):
    """||PA - LU||_F / ||A||_F <= 20 n 2^-53, valid swap sequence, unit L,
    and |L| bounded (Section 7.3 cites tournament pivoting as stable as
    partial pivoting; the bound 32 is this build's reading)."""
    A = wl.matrix_uniform(m, n, seed=m * 7 + n)
    LU, piv, info = oracle_mod.lu_factor(A, b=b, h=h)
    assert info == 0
    k = min(m, n)
    assert ((piv >= np.arange(k)) & (piv < m)).all()
    L, U = split_lu(LU)
    PA = apply_piv(A, piv)
    res = np.linalg.norm(PA - L @ U) / np.linalg.norm(A)
    assert res <= 20 * max(m, n) * EPS, res
    assert np.abs(L).max() <= 32.0


# --- loop bounds of Section 6 ----------------------------------------------

@pytest.mark.parametrize("n,b,h", [(1, 1, 1), (2, 1, 1), (4, 2, 2), (17, 4, 3), (64, 8, 16), (63, 16, 4)])
def test_vertex_counts(oracle_mod, n, b, h):
    """The oracle performs exactly sum_{i,j} min(i,j) = n^3/3 - n^2/2 + n/6
    fused S2 updates and n(n-1)/2 S1 divisions on the matrix.  The paper's
    |V_S2| = N^3/3 - N^2 + 2N/3 (Section 6) counts N(N-1)/2 fewer: its sums
    run to N-k-1, the same off-by-one as its |V_S1| sum."""
    A = wl.matrix_uniform(n, n, seed=1)
    _, _, _, (s1, s2) = oracle_mod.lu_factor(A, b=b, h=h, count=True)
    assert 6 * s2 == 2 * n ** 3 - 3 * n ** 2 + n
    assert 2 * s1 == n * (n - 1)
    paper_vs2 = Fraction(n ** 3, 3) - n ** 2 + Fraction(2 * n, 3)
    assert s2 - paper_vs2 == Fraction(n * (n - 1), 2)


@pytest.mark.parametrize("m,n", [(10, 6), (6, 10), (33, 20)])
def test_vertex_counts_rectangular(oracle_mod, m, n):
    """m x n: each element (i, j) gets min(i, j, min(m,n)) updates."""
    A = wl.matrix_uniform(m, n, seed=2)
    _, _, _, (s1, s2) = oracle_mod.lu_factor(A, b=4, h=3, count=True)
    k = min(m, n)
    expect = sum(min(i, j, k) for i in range(m) for j in range(n))
    assert s2 == expect
    assert s1 == sum(m - 1 - j for j in range(k))


def test_paper_counts_golden(oracle_mod):
    """tests/golden/paper_counts.txt: the Section 6 formulas at the N = 4 of
    Fig. 1, with the oracle's count beside them."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            key, val = line.split("=")
            rows[key.strip()] = int(val)
    N = rows["N"]
    assert Fraction(N ** 3, 3) - N ** 2 + Fraction(2 * N, 3) == rows["paper_VS2"]
    assert Fraction(N * (N - 1), 2) == rows["paper_VS1"]
    A = wl.matrix_uniform(N, N, seed=0)
    _, _, _, (s1, s2) = oracle_mod.lu_factor(A, b=1, h=1, count=True)
    assert s2 == rows["updates_S2"]
    assert s1 == rows["divisions_S1"]


# --- brute force with exact rationals ----------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_exact_rational_tournament(oracle_mod, n):
    """Pivots of the binary64 oracle equal those of an independent exact
    rational restatement for every b in {1,2,3} and h in {1,2,4}."""
    for seed in range(4):
        A = wl.matrix_uniform(n, n, seed=300 + seed, stream=n)
        for b, h in itertools.product([1, 2, 3], [1, 2, 4]):
            _, piv, info = oracle_mod.lu_factor(A, b=b, h=h)
            M, piv_x = exact_lu(A.tolist(), b, h)
            assert list(piv) == piv_x, (n, seed, b, h)
            LU, _, _ = oracle_mod.lu_factor(A, b=b, h=h)
            Mx = np.array([[float(x) for x in row] for row in M])
            np.testing.assert_allclose(LU, Mx, rtol=0, atol=1e-12 * max(1.0, np.abs(Mx).max()))


@pytest.mark.parametrize("m,w,h", [(8, 2, 1), (9, 3, 2), (12, 4, 3), (7, 2, 4)])
def test_exact_tslu_select(oracle_mod, m, w, h):
    """One TournPivot call (winners in root order) against exact rationals,
    on a panel in the middle of the matrix (k > 0)."""
    from tests.exact_tournament import tournament
    A = wl.matrix_normal(m, m, seed=m, stream=w)
    k = 1
    win = oracle_mod.tslu_select(A, k=k, w=w, h=h)
    M = [[Fraction(x) for x in row] for row in A.tolist()]
    assert list(win) == tournament(M, k, w, h)


# --- solve and backward error -------------------------------------------------

@pytest.mark.parametrize("n,nrhs", [(1, 1), (10, 3), (120, 1), (200, 8)])
def test_solve_matches_numpy(oracle_mod, n, nrhs):
    A = wl.matrix_uniform(n, n, seed=n)
    B = wl.matrix_uniform(n, nrhs, seed=n + 1)
    LU, piv, info = oracle_mod.lu_factor(A, b=16, h=8)
    X = oracle_mod.lu_solve(LU, piv, B)
    Xr = np.linalg.solve(A, B)
    cond = np.linalg.cond(A)
    assert np.abs(X - Xr).max() <= 1e3 * cond * EPS * np.abs(Xr).max()


def test_solve_exact_integer_system(oracle_mod):
    """Unit upper triangular integer system and its permutation: exact."""
    n = 9
    U = np.triu(np.ones((n, n)))
    x = np.arange(1, n + 1, dtype=np.float64)
    b = U @ x
    LU, piv, info = oracle_mod.lu_factor(U, b=4, h=2)
    np.testing.assert_array_equal(oracle_mod.lu_solve(LU, piv, b), x)


def test_backward_error_closed_forms(oracle_mod):
    """eta = 0 for an exact solution; a hand-computed 2 x 2 case."""
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    x = np.array([1.0, -1.0])
    b = A @ x
    assert oracle_mod.backward_error(A, b, x)[0] == 0.0
    xp = np.array([1.0, -0.5])          # r = b - A xp = [-0.5, -1.5]
    # ||r||=1.5, ||A||_inf = 4, ||xp|| = 1, ||b|| = 2  ->  1.5 / 6
    assert oracle_mod.backward_error(A, b, xp)[0] == 0.25


@pytest.mark.parametrize("n", [4, 5, 6])
def test_ties_go_to_smallest_position(oracle_mod, n):
    """Entries in {-1, 0, 1} make exact ties common.  Wherever the binary64
    run is exact (it equals the rational factors), the pivots must equal the
    exact tournament's, whose tie rule is 'smallest row position'."""
    checked = 0
    for seed in range(40):
        u = wl.uniform01(700 + n, seed, np.arange(n * n, dtype=np.uint64))
        M = (np.floor(u * 3) - 1).reshape(n, n)
        for b, h in [(1, 1), (2, 1), (2, 2), (3, 2)]:
            LU, piv, info = oracle_mod.lu_factor(M, b=b, h=h)
            Mx, piv_x = exact_lu(M.tolist(), b, h)
            if any(float(x) != y for rx, ry in zip(Mx, LU.tolist()) for x, y in zip(rx, ry)):
                continue
            if any(Fraction(float(x)) != x for row in Mx for x in row):
                continue
            assert list(piv) == piv_x, (M, b, h)
            checked += 1
    assert checked >= 40


def test_first_column_tie(oracle_mod):
    """|A[:,0]| all equal: the first pivot is row 0 (smallest position), as
    in LAPACK idamax; a 'last maximum' rule would pick another row."""
    n = 40
    A = wl.matrix_uniform(n, n, seed=77)
    A[:, 0] = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
    for b, h in [(1, 4), (8, 4), (8, 64)]:
        _, piv, _ = oracle_mod.lu_factor(A, b=b, h=h)
        assert piv[0] == 0
    _, ipiv = sla.lu_factor(A)
    assert ipiv[0] == 0


@pytest.mark.parametrize("n,b,h", [(10, 2, 1), (13, 3, 2), (16, 4, 1), (16, 2, 3), (11, 5, 1)])
def test_exact_rational_deeper_trees(oracle_mod, n, b, h):
    """Trees four or more levels deep (many leaves, selection at several
    levels) against the exact rational restatement: pins the leaf cut, the
    pairing of adjacent nodes and the promotion of an odd last node."""
    for seed in range(3):
        A = wl.matrix_uniform(n, n, seed=900 + seed, stream=n * 10 + h)
        _, piv, _ = oracle_mod.lu_factor(A, b=b, h=h)
        _, piv_x = exact_lu(A.tolist(), b, h)
        assert list(piv) == piv_x, (n, b, h, seed)
