"""An exact-rational restatement of tournament-pivoting LU for tiny inputs.

Written independently of the C oracle (recursive tree over row ranges, exact
Fractions instead of binary64) so that it can pin the oracle's tree shape,
pairing order, tie rule and swap bookkeeping on n <= 8.  Test helper only.
"""
from __future__ import annotations

from fractions import Fraction


def _select(M, rows, k, w):
    """Local LUP on the given row positions over panel columns k..k+w-1;
    returns min(len(rows), w) positions in pivot order (exact arithmetic)."""
    work = {r: [Fraction(M[r][k + j]) for j in range(w)] for r in rows}
    remaining = list(rows)
    chosen = []
    for c in range(min(len(rows), w)):
        # largest |value|; equal values go to the smallest position
        best = min(remaining, key=lambda r: (-abs(work[r][c]), r))
        chosen.append(best)
        remaining.remove(best)
        p = work[best][c]
        if p != 0:
            for r in remaining:
                f = work[r][c] / p
                for j in range(c, w):
                    work[r][j] -= f * work[best][j]
    return chosen


def _node(M, k, w, h, lo, hi, first_leaf, nleaf_span):
    """Candidates of the node covering leaves [first_leaf, first_leaf+span)."""
    r0 = k + first_leaf * h
    r1 = min(hi, r0 + nleaf_span * h)
    if nleaf_span == 1:
        return _select(M, list(range(r0, r1)), k, w)
    half = nleaf_span // 2
    left = _node(M, k, w, h, lo, hi, first_leaf, half)
    right_first = first_leaf + half
    if k + right_first * h >= hi:
        return left
    right = _node(M, k, w, h, lo, hi, right_first, half)
    return _select(M, left + right, k, w)


def tournament(M, k, w, h):
    """Winners over active rows [k, m) as a recursive tree of leaves of h."""
    m = len(M)
    nleaf = (m - k + h - 1) // h
    span = 1
    while span < nleaf:
        span *= 2
    return _node(M, k, w, h, k, m, 0, span)


def lu(A, b, h):
    """Returns (LU as Fractions, piv) for the blocked tournament LU."""
    M = [[Fraction(x) for x in row] for row in A]
    m, n = len(M), len(M[0])
    piv = []
    for k in range(0, min(m, n), b):
        w = min(b, min(m, n) - k)
        win = tournament(M, k, w, h)
        # move each winner, in order, to the next top row by one swap,
        # tracking where every row identity currently sits
        ident = list(range(m))
        pos = {r: r for r in range(m)}
        for j, r in enumerate(win):
            p = pos[r]
            piv.append(p)
            a, bb = k + j, p
            M[a], M[bb] = M[bb], M[a]
            ra, rb = ident[a], ident[bb]
            ident[a], ident[bb] = rb, ra
            pos[rb], pos[ra] = a, bb
        # eliminate the block column by column (exact, any order)
        for j in range(k, k + w):
            d = M[j][j]
            for i in range(j + 1, m):
                f = M[i][j] / d if d != 0 else Fraction(0)
                M[i][j] = f
                if f != 0:
                    for c in range(j + 1, n):
                        M[i][c] -= f * M[j][c]
    return M, piv
