"""Exact rational Moore-Penrose inverse for tiny integer matrices.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and by the script that writes
``tests/golden/``).  Pure-Python ``fractions.Fraction`` arithmetic, so the
result is the exact G+ of Sec. 1, with no rounding at all.

Route (independent of the Cholesky route of the Appendix): a full-rank
factorisation G = C F from the reduced row-echelon form -- C holds the pivot
columns of G (m x r), F the non-zero rows of the RREF (r x n) -- and then

    G+ = F' (F F')^-1 (C'C)^-1 C'

which is Eq. (4) of Sec. 2 applied to each factor together with Eq. (2)
(the reverse-order law holds for a full-column-rank C times a full-row-rank F).
"""
from __future__ import annotations

from fractions import Fraction


def _mat(rows):
    return [[Fraction(x) for x in row] for row in rows]


def _transpose(A):
    return [list(col) for col in zip(*A)] if A else []


def _matmul(A, B):
    if not A or not B:
        return [[Fraction(0)] * (len(B[0]) if B else 0) for _ in A]
    Bt = _transpose(B)
    return [[sum((a * b for a, b in zip(row, col)), Fraction(0)) for col in Bt] for row in A]


def _inverse(A):
    """Gauss-Jordan inverse of a non-singular square Fraction matrix."""
    n = len(A)
    M = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    return [row[n:] for row in M]


def rref(A):
    """Reduced row-echelon form and the pivot column indices."""
    R = [row[:] for row in A]
    m = len(R)
    n = len(R[0]) if m else 0
    pivots = []
    row = 0
    for c in range(n):
        p = next((i for i in range(row, m) if R[i][c] != 0), None)
        if p is None:
            continue
        R[row], R[p] = R[p], R[row]
        piv = R[row][c]
        R[row] = [x / piv for x in R[row]]
        for i in range(m):
            if i != row and R[i][c] != 0:
                f = R[i][c]
                R[i] = [a - f * b for a, b in zip(R[i], R[row])]
        pivots.append(c)
        row += 1
        if row == m:
            break
    return R, pivots


def exact_pinv(G_int):
    """Exact G+ (list of lists of Fraction, n x m) of an integer/rational G."""
    G = _mat(G_int)
    m = len(G)
    n = len(G[0]) if m else 0
    R, piv = rref(G)
    r = len(piv)
    if r == 0:
        return [[Fraction(0)] * m for _ in range(n)]
    C = [[G[i][j] for j in piv] for i in range(m)]          # m x r
    F = R[:r]                                               # r x n
    Ct = _transpose(C)
    Ft = _transpose(F)
    left = _matmul(Ft, _inverse(_matmul(F, Ft)))            # n x r
    right = _matmul(_inverse(_matmul(Ct, C)), Ct)           # r x m
    return _matmul(left, right)


def exact_rank(G_int) -> int:
    return len(rref(_mat(G_int))[1])
