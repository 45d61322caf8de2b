"""Plain FP64 CPU oracle of the full-rank-Cholesky Moore-Penrose inverse.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU legs of ``bench.py`` (the timed
``cpu_baseline`` sample and ``--impl reference``).  The library path never
imports it and shares no code, table or helper with it.

What it computes (Courrieu, "Fast Computation of Moore-Penrose Inverse
Matrices"):

* Sec. 1: the Moore-Penrose inverse G+ of a real m x n matrix G, defined by the
  four Penrose conditions, and the least-squares weights W = G+ F (the printed
  "W = G+ W" is read as W = G+ F, since F is the target matrix of the problem
  statement).
* Sec. 2, Eq. (1) and Theorem 1: G'G = L L' with L (n x r) of full column rank
  r, and G+ = L (L'L)^-1 (L'L)^-1 L' G'.
* Appendix (function ``geninv``): the steps below, in the paper's order --
  transpose when m < n; A = G'G (rounded once per entry, see ``gram``); tol = 1e-9 * (smallest positive diagonal
  entry of A); left-looking full-rank Cholesky in natural column order, a
  column being kept when its updated pivot is strictly above tol; L trimmed to
  its r kept columns; M = inv(L'L); Y = L M M L' G' evaluated left to right.

Library primitives serve as single steps (a matrix product, a matrix-vector
product, ``numpy.linalg.inv`` = LU with partial pivoting like Matlab's
``inv``); there is no blocking or reordering beyond the algorithm's own.

Reading of the Appendix listing (see ``full_rank_cholesky``): when a pivot is
rejected, the listing leaves the rejected residual in row k of the column that
the next kept pivot will occupy.  Theorem 1 needs S with *exactly* zero rows
(Sec. 2), i.e. column j of L zero above its pivot row.  The default here keeps
that zero (theorem semantics); ``literal=True`` reproduces the listing.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against independent facts (Penrose conditions, exact rational arithmetic, a
hand-written Jacobi SVD, a Householder-QR closed form, special cases with
closed forms).
"""
from __future__ import annotations

import math

import numpy as np

#: Appendix: the pivot threshold is this factor times the smallest positive
#: diagonal entry of A = G'G (an absolute threshold, not scaled by n or eps).
REL_TOL = 1e-9


def _two_sum(a, b):
    """Error-free transformation (Knuth): s + e == a + b exactly."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def exact_cross(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X'Y with every entry equal to the exact dot product rounded once to FP64.

    Route: scale each column by a power of two so |x| <= 1; cut it into
    integer slices of ``b`` bits (x = sum_s d_s 2^(-b(s+1)) + a remainder
    below 2^(-b S), with S b >= 72); every slice product D_s'D_t has integer
    partial sums below 2^53 (b <= (53 - log2 m) / 2), so the FP64 matrix
    product computes it exactly in any summation order; the exact terms are
    then added with an error-free (double-double) accumulation from the
    smallest weight up and rounded once.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    m = X.shape[0]
    if m == 0 or X.shape[1] == 0 or Y.shape[1] == 0:
        return np.zeros((X.shape[1], Y.shape[1]))
    b = (53 - max(1, math.ceil(math.log2(m)))) // 2
    S = -(-72 // b)

    def split(Z):
        amax = np.max(np.abs(Z), axis=0)
        e = np.zeros(Z.shape[1], dtype=np.int64)
        nz = amax > 0
        e[nz] = np.ceil(np.log2(amax[nz])).astype(np.int64)
        R = Z * np.ldexp(1.0, -e)[None, :]
        D = []
        for s in range(S):
            w = math.ldexp(1.0, b * (s + 1))
            d = np.trunc(R * w)
            D.append(d)
            R = R - d / w
        return D, e

    DX, ex = split(X)
    DY, ey = split(Y)
    hi = np.zeros((X.shape[1], Y.shape[1]))
    lo = np.zeros_like(hi)
    for T in range(2 * S - 2, -1, -1):           # smallest weights first
        for s in range(S):
            t = T - s
            if 0 <= t < S:
                P = (DX[s].T @ DY[t]) * math.ldexp(1.0, -b * (T + 2))
                hi, err = _two_sum(hi, P)
                lo += err
    A = hi + lo
    return A * np.ldexp(1.0, ex[:, None] + ey[None, :])


def gram(G: np.ndarray, exact: bool = True) -> np.ndarray:
    """A = G'G (Appendix; Sec. 2, Eq. (1)).  n x n, FP64.

    ``exact=True`` (default): each entry is the exact inner product of two
    columns rounded once (``exact_cross``).  ``exact=False``: the FP64 matrix
    product with the BLAS library's own rounding order.  The
    paper does not fix the rounding of G'G; the method's G+ moves by about
    1e-10 (relative) between two FP64 summation orders on rank-deficient
    Gaussian products, so the oracle takes the one rounding that does not
    depend on an implementation.
    """
    G = np.asarray(G, dtype=np.float64)
    if exact:
        return exact_cross(G, G)
    return G.T @ G


def pivot_tolerance(A: np.ndarray, rel_tol: float = REL_TOL):
    """tol = rel_tol * min{A_jj : A_jj > 0} (Appendix).

    Returns ``None`` when no diagonal entry is positive: Matlab's
    ``min([])`` is empty, every ``L(k,r) > tol`` test is then false and the
    rank is 0.
    """
    dA = np.diag(A)
    pos = dA[dA > 0]
    if pos.size == 0:
        return None
    return float(pos.min()) * rel_tol


def full_rank_cholesky(A: np.ndarray, tol, literal: bool = False, keep=None):
    """Full-rank Cholesky of a symmetric positive semidefinite A (Appendix).

    Natural column order, no pivoting.  For k = 0..n-1, with r columns kept
    so far, the candidate column is

        v = A[k:, k] - L[k:, :r] @ L[k, :r]

    and it is kept iff ``v[0] > tol`` (strict; NaN is rejected): then
    ``L[k, r] = sqrt(v[0])`` and ``L[k+1:, r] = v[1:] / L[k, r]``.

    Returns ``(L, accepted, pivots)``: L is n x r (the kept columns, in
    order), ``accepted`` the boolean mask of kept pivot indices and
    ``pivots[k]`` the candidate value v[0] tested at step k.

    ``keep`` (a boolean mask) replaces the pivot test by a given kept set:
    the same function with S held fixed, whose derivative is the method's
    derivative (``oracle.adjoint``).  A forced pivot must be positive.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros((n, n), dtype=np.float64)
    accepted = np.zeros(n, dtype=bool)
    pivots = np.zeros(n, dtype=np.float64)
    r = 0
    for k in range(n):
        # candidate column k: column k of A minus the contribution of the r
        # columns kept so far (left-looking update, Sec. 2 Eq. (1))
        v = A[k:, k] - L[k:, :r] @ L[k, :r]
        pivots[k] = v[0]
        if (keep[k] and v[0] > 0) if keep is not None else (tol is not None and v[0] > tol):
            d = math.sqrt(v[0])
            L[k, r] = d
            if k + 1 < n:
                L[k + 1:, r] = v[1:] / d
            accepted[k] = True
            r += 1
        elif literal and r < n:
            # The listing wrote v into column r before testing it; rows
            # k+1.. are overwritten by the next candidate, row k is not.
            L[k:, r] = v
    return L[:, :r].copy(), accepted, pivots


def geninv(G: np.ndarray, rel_tol: float = REL_TOL, literal: bool = False,
           return_factors: bool = False, exact_gram: bool = True, keep=None):
    """Moore-Penrose inverse of any real rectangular G (Appendix ``geninv``).

    Returns Y = G+ (n x m).  With ``return_factors`` also returns a dict with
    the rank r, the accepted mask, L, M = inv(L'L), tol and whether the
    transposed branch (m < n, A = G G') was taken.  ``keep`` forces the
    kept-pivot set (see ``full_rank_cholesky``).
    """
    G = np.asarray(G, dtype=np.float64)
    if G.ndim != 2:
        raise ValueError("G must be 2-D")
    m, n = G.shape
    transpose = m < n
    # Appendix: the wide case (m < n) factors G G' of order m instead.
    A = gram(G.T if transpose else G, exact=exact_gram)
    nA = A.shape[0]
    if nA == 0:
        Y = np.zeros((n, m))
        fac = dict(rank=0, accepted=np.zeros(0, bool), L=np.zeros((0, 0)),
                   M=np.zeros((0, 0)), tol=None, transpose=transpose)
        return (Y, fac) if return_factors else Y
    tol = pivot_tolerance(A, rel_tol)
    L, accepted, pivots = full_rank_cholesky(A, tol, literal=literal, keep=keep)
    r = L.shape[1]
    if r == 0:
        M = np.zeros((0, 0))
        Y = np.zeros((n, m))
    else:
        M = np.linalg.inv(L.T @ L)
        # Matlab evaluates the chain left to right; so does numpy's '@'.
        if transpose:
            Y = G.T @ L @ M @ M @ L.T
        else:
            Y = L @ M @ M @ L.T @ G.T
    if return_factors:
        return Y, dict(rank=r, accepted=accepted, pivots=pivots, L=L, M=M,
                       tol=tol, transpose=transpose)
    return Y


def rank(G: np.ndarray, rel_tol: float = REL_TOL, exact_gram: bool = True):
    """Numerical rank r and accepted-pivot mask of the Appendix factorisation."""
    _, fac = geninv(G, rel_tol=rel_tol, return_factors=True, exact_gram=exact_gram)
    return fac["rank"], fac["accepted"]


def lstsq(G: np.ndarray, F: np.ndarray, rel_tol: float = REL_TOL,
          exact_gram: bool = True, keep=None) -> np.ndarray:
    """Minimum-norm least-squares weights W = G+ F (Sec. 1; the printed
    ``W = G+ W`` read as ``W = G+ F``)."""
    F = np.asarray(F, dtype=np.float64)
    return geninv(G, rel_tol=rel_tol, exact_gram=exact_gram, keep=keep) @ F


def lstsq_from_gram(A: np.ndarray, B: np.ndarray, rel_tol: float = REL_TOL) -> tuple:
    """W = L M M L' B from given normal equations A = G'G, B = G'F (Appendix
    steps from the Gram matrix on; Theorem 1 with L' G' F = L' B).  The
    method needs G only through A and B, which is what makes accumulating
    them block by block possible (Sec. 4: on-line and incremental learning).
    Only the lower triangle of A is read.  Returns (W, rank)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    A = np.tril(A) + np.tril(A, -1).T
    tol = pivot_tolerance(A, rel_tol)
    L, accepted, _ = full_rank_cholesky(A, tol)
    r = L.shape[1]
    if r == 0:
        return np.zeros((A.shape[0], B.shape[1])), 0
    M = np.linalg.inv(L.T @ L)
    return L @ M @ M @ L.T @ B, r


def penrose_residuals(G: np.ndarray, Y: np.ndarray) -> dict:
    """The four Penrose error matrices of Sec. 1 / Sec. 3, as max-abs and
    Frobenius norms: GYG - G, YGY - Y, (GY)' - GY, (YG)' - YG."""
    G = np.asarray(G, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    GY = G @ Y
    YG = Y @ G
    mats = {
        "GYG-G": GY @ G - G,
        "YGY-Y": Y @ GY - Y,
        "sym(GY)": GY.T - GY,
        "sym(YG)": YG.T - YG,
    }
    out = {}
    for k, E in mats.items():
        out[k + ":max"] = float(np.max(np.abs(E))) if E.size else 0.0
        out[k + ":fro"] = float(np.linalg.norm(E)) if E.size else 0.0
    return out
