"""Reverse-mode derivative of the least-squares weights W = G+ F computed by
the method (FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY (same rules as ``oracle.geninv``: imported by the
tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``; shares no
code with the library).

The paper does not differentiate its method; this is the derivative of the
function the Appendix computes, with the kept-pivot set S held fixed (the
rank decision is piecewise constant, so that is its derivative wherever it
exists).  With S fixed the method is a composition of smooth steps, taken
here in the forward order of ``oracle.geninv`` and reversed one by one:

  A  = G'G                                      (Appendix; Eq. (1))
  L  = full-rank Cholesky factor of A on S      (Appendix)
  N  = L'L,   M = N^-1                          (Theorem 1)
  B  = G'F,  c1 = L'B,  c2 = M c1,  c3 = M c2,  W = L c3
                                                (Theorem 1 applied to F)

The factor L (n x r, columns = kept pivots in order) has, in the row of
column index i and the column of kept pivot s_c, a structural zero whenever
s_c > i: the natural-order algorithm fills column c only from its pivot row
down (rows of rejected pivots included).  Its rows split into the kept rows
S, which form the lower-triangular L_S with L_S L_S' = A_SS, and the
rejected rows D, with L_D = (A_DS L_S^-T) restricted to that pattern.  The
adjoints of the two pieces (for a lower-triangular Cholesky factor, the
standard result Abar = L^-T Phi(L' Lbar) L^-1, Phi = lower triangle with the
diagonal halved):

  Lbar_D <- Lbar_D on the pattern,   Abar_DS = Lbar_D L_S^-1,
  Lbar_S <- Lbar_S - L_S^-T Lbar_D' L_D,
  Abar_SS = L_S^-T Phi(L_S' Lbar_S) L_S^-1,   Abar_DD = Abar_SD = 0.

Every dense step is a library matrix product or a triangular solve
(``numpy.linalg.solve`` on the triangular factor).  When m < n the method
works on H = G' (A = G G'); the derivative is taken through that branch and
transposed back.
"""
from __future__ import annotations

import numpy as np

from .geninv import REL_TOL, full_rank_cholesky, gram, pivot_tolerance


def _phi(X: np.ndarray) -> np.ndarray:
    """Lower triangle of X with the diagonal halved."""
    P = np.tril(X)
    P[np.diag_indices_from(P)] *= 0.5
    return P


def _forward(G: np.ndarray, F: np.ndarray, rel_tol: float, exact_gram: bool, keep=None):
    """The forward quantities of the method for W = G+ F, m >= n."""
    A = gram(G, exact=exact_gram)
    tol = pivot_tolerance(A, rel_tol)
    L, accepted, _ = full_rank_cholesky(A, tol, keep=keep)
    N = L.T @ L
    M = np.linalg.inv(N) if L.shape[1] else np.zeros((0, 0))
    M = 0.5 * (M + M.T)
    B = G.T @ F
    c1 = L.T @ B
    c2 = M @ c1
    c3 = M @ c2
    W = L @ c3
    return dict(A=A, L=L, accepted=accepted, M=M, B=B, c1=c1, c2=c2, c3=c3, W=W)


def lstsq_vjp(G: np.ndarray, F: np.ndarray, dW: np.ndarray, rel_tol: float = REL_TOL,
              exact_gram: bool = True, keep=None):
    """(W, dG, dF) for W = G+ F and the cotangent dW (n x k): dG = dL/dG and
    dF = dL/dF for any scalar L with dL/dW = dW, S held fixed (the pivot
    test's, or ``keep`` when given)."""
    G = np.asarray(G, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    dW = np.asarray(dW, dtype=np.float64)
    m, n = G.shape
    if m < n:
        return _vjp_transposed(G, F, dW, rel_tol, exact_gram, keep)
    fw = _forward(G, F, rel_tol, exact_gram, keep)
    L, M, B = fw["L"], fw["M"], fw["B"]
    c1, c2, c3 = fw["c1"], fw["c2"], fw["c3"]
    acc = fw["accepted"]
    r = L.shape[1]
    if r == 0:
        return fw["W"], np.zeros_like(G), np.zeros_like(F)

    # chain W = L c3, c3 = M c2, c2 = M c1, c1 = L'B, B = G'F
    Lbar = dW @ c3.T
    c3bar = L.T @ dW
    Mbar = c3bar @ c2.T
    c2bar = M @ c3bar
    Mbar += c2bar @ c1.T
    c1bar = M @ c2bar
    Lbar += B @ c1bar.T
    Bbar = L @ c1bar

    # M = N^-1, N = L'L
    Nbar = -M @ Mbar @ M
    Lbar += L @ (Nbar + Nbar.T)

    # full-rank Cholesky with S fixed
    S = np.flatnonzero(acc)
    D = np.flatnonzero(~acc)
    pattern = S[None, :] <= np.arange(n)[:, None]   # (i, c) kept iff s_c <= i
    Lbar = Lbar * pattern
    LS, LD = L[S, :], L[D, :]
    LbS, LbD = Lbar[S, :], Lbar[D, :]
    Abar = np.zeros((n, n))
    if D.size:
        # Abar_DS = LbD LS^-1  <=>  LS' Abar_DS' = LbD'
        Abar[np.ix_(D, S)] = np.linalg.solve(LS.T, LbD.T).T
        LbS = LbS - np.linalg.solve(LS.T, LbD.T @ LD)
    P = _phi(LS.T @ LbS)
    # Abar_SS = LS^-T P LS^-1
    Y = np.linalg.solve(LS.T, P)                    # LS^-T P
    Abar[np.ix_(S, S)] = np.linalg.solve(LS.T, Y.T).T  # (LS^-T (LS^-T P)')' = LS^-T P LS^-1

    # A = G'G, B = G'F
    dG = G @ (Abar + Abar.T) + F @ Bbar.T
    dF = G @ Bbar
    return fw["W"], dG, dF


def _vjp_transposed(G, F, dW, rel_tol, exact_gram, keep=None):
    """m < n: the Appendix factors A = G G' (H = G', m x m Gram) and returns
    G+ = (H+)'; W = G+ F = G' (L M M L') F with L from A = H'H.  Chain:
    c1 = L'F, c2 = M c1, c3 = M c2, t = L c3, W = G' t."""
    H = G.T                                           # n x m, tall
    A = gram(H, exact=exact_gram)
    tol = pivot_tolerance(A, rel_tol)
    L, acc, _ = full_rank_cholesky(A, tol, keep=keep)
    mA = A.shape[0]
    r = L.shape[1]
    if r == 0:
        return np.zeros((G.shape[1], F.shape[1])), np.zeros_like(G), np.zeros_like(F)
    M = np.linalg.inv(L.T @ L)
    M = 0.5 * (M + M.T)
    c1 = L.T @ F
    c2 = M @ c1
    c3 = M @ c2
    t = L @ c3
    W = G.T @ t
    # W = G' t
    dG = t @ dW.T                                     # m x n
    tbar = G @ dW
    # t = L c3, ...
    Lbar = tbar @ c3.T
    c3bar = L.T @ tbar
    Mbar = c3bar @ c2.T
    c2bar = M @ c3bar
    Mbar += c2bar @ c1.T
    c1bar = M @ c2bar
    Lbar += F @ c1bar.T
    dF = L @ c1bar
    Nbar = -M @ Mbar @ M
    Lbar += L @ (Nbar + Nbar.T)
    S = np.flatnonzero(acc)
    D = np.flatnonzero(~acc)
    pattern = S[None, :] <= np.arange(mA)[:, None]
    Lbar = Lbar * pattern
    LS, LD = L[S, :], L[D, :]
    LbS, LbD = Lbar[S, :], Lbar[D, :]
    Abar = np.zeros((mA, mA))
    if D.size:
        Abar[np.ix_(D, S)] = np.linalg.solve(LS.T, LbD.T).T
        LbS = LbS - np.linalg.solve(LS.T, LbD.T @ LD)
    P = _phi(LS.T @ LbS)
    Y = np.linalg.solve(LS.T, P)
    Abar[np.ix_(S, S)] = np.linalg.solve(LS.T, Y.T).T
    # A = H'H = G G': dA = dG G' + G dG'  ->  dG += (Abar + Abar') G
    dG += (Abar + Abar.T) @ G
    return W, dG, dF


def golub_pereyra_vjp(G: np.ndarray, F: np.ndarray, dW: np.ndarray, Gp: np.ndarray):
    """Golub & Pereyra (1973): the derivative of G+ along perturbations of
    constant rank, dG+ = -G+ dG G+ + G+ G+' dG' (I - G G+) + (I - G+ G) dG'
    G+' G+, pulled back through W = G+ F:

      dG = -G+' dW W' + (F - G W) dW' G+ G+' + G+' W dW' (I - G+ G).

    ``Gp`` is G+ (any correct one).  Used as an independent check of
    ``lstsq_vjp`` on inputs of exact rank."""
    W = Gp @ F
    n = G.shape[1]
    R = F - G @ W
    return (-Gp.T @ dW @ W.T + R @ dW.T @ Gp @ Gp.T
            + Gp.T @ W @ dW.T @ (np.eye(n) - Gp @ G))
