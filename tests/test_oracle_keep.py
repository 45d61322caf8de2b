"""Pins of the oracle's forced kept-set branch (``keep=``).

The GPU tests compare the least-squares weights and the adjoint of RBF
workloads for the GPU's own kept set S (the rank decision of an RBF Gram
matrix is not stable between two FP64-class evaluations), so the oracle's
``full_rank_cholesky(..., keep=)`` must be right on its own.  It is pinned
here by facts that do not come from the oracle:

* with its own accepted mask forced, the oracle reproduces itself bit for
  bit (same operations, same order);
* the factor for a forced S, computed another way: its rows in S are the
  Cholesky factor of A_SS (LAPACK's Cholesky here), and a row d outside S
  holds A[d, V] L_V^-T in the columns of the kept pivots V before d (a
  triangular solve with the leading block) and zeros after (each column is
  filled from its own pivot row down);
* when every dropped column precedes the kept ones, the dropped rows of L are
  zero and G+ reduces to the pseudoinverse of G[:, S] scattered back (rows
  outside S zero), checked against a Householder-QR closed form;
* a forced pivot that is not positive is still rejected (exactly repeated
  integer columns, against the exact rational G+);
* planted mistakes in a copy of the forced branch are each caught.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.exact import exact_pinv
from oracle.geninv import full_rank_cholesky, geninv, pivot_tolerance
from oracle.jacobi import jacobi_svd_pinv
from paper_0804_4809_gb300 import inputs


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _forced_factor(A, S):
    """The forced-set factor without the left-looking loop: LAPACK's
    Cholesky of A_SS for the rows in S; for a row d outside S, the kept
    pivots V before d give L[d, V] = A[d, V] L_S[V, V]^-T (V is a prefix of S,
    so L_S[V, V] is a leading block), zeros after."""
    n = A.shape[0]
    S = np.asarray(S)
    LS = np.linalg.cholesky(A[np.ix_(S, S)])
    L = np.zeros((n, len(S)))
    L[S] = LS
    for d in np.setdiff1d(np.arange(n), S):
        v = int(np.sum(S < d))
        if v:
            L[d, :v] = np.linalg.solve(LS[:v, :v], A[d, S[:v]])
    return L


def _theorem1(L, G):
    """L (L'L)^-1 (L'L)^-1 L' G' by two linear solves."""
    N = L.T @ L
    return L @ np.linalg.solve(N, np.linalg.solve(N, L.T @ G.T))


def _qr_pinv(H):
    Q, R = np.linalg.qr(H)
    return np.linalg.solve(R, Q.T)


@pytest.mark.parametrize("which", ["small", "paper64", "paper128"])
def test_own_mask_reproduces_geninv_bit_for_bit(which):
    if which == "small":
        G = inputs.workload_small()
    else:
        n = int(which[5:])
        G = inputs.paper_family(n, seed=n)
    Y, fac = geninv(G, return_factors=True)
    Yk, fk = geninv(G, return_factors=True, keep=fac["accepted"])
    assert fk["rank"] == fac["rank"]
    assert np.array_equal(fk["accepted"], fac["accepted"])
    assert np.array_equal(fk["L"], fac["L"])
    assert np.array_equal(Yk, Y)
    F = inputs.normal((G.shape[0], 3), seed=5)
    assert np.array_equal(oracle.lstsq(G, F, keep=fac["accepted"]), oracle.lstsq(G, F))


def _forced_set(n, S):
    keep = np.zeros(n, dtype=bool)
    keep[list(S)] = True
    return keep


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_forced_factor_matches_independent_route(seed):
    """Random forced sets on full-rank and rank-deficient inputs: the
    oracle's factor equals the one built from LAPACK's Cholesky and
    triangular solves, and its G+ equals Theorem 1's formula for that
    factor."""
    rng = np.random.default_rng(seed)
    for G in (inputs.full_rank(60, 14, seed=seed), inputs.rank_deficient(70, 16, 12, seed)):
        A = oracle.gram(G)
        n = A.shape[0]
        S = np.sort(rng.choice(n, size=8, replace=False))
        assert np.linalg.matrix_rank(G[:, S]) == 8
        Y, fac = geninv(G, return_factors=True, keep=_forced_set(n, S))
        assert np.array_equal(np.flatnonzero(fac["accepted"]), S)
        Lx = _forced_factor(A, S)
        assert _rel(fac["L"], Lx) < 1e-12, _rel(fac["L"], Lx)
        assert _rel(Y, _theorem1(Lx, G)) < 1e-10


@pytest.mark.parametrize("m,n,r,seed", [(60, 30, 18, 4), (45, 20, 11, 5), (50, 12, 12, 6)])
def test_suffix_set_gives_pinv_of_the_kept_columns(m, n, r, seed):
    """Every dropped column before the kept ones: the dropped rows of L stay
    zero, so G+ is the pseudoinverse of G[:, S] with zero rows outside S."""
    G = inputs.rank_deficient(m, n, r, seed) if r < n else inputs.full_rank(m, n, seed)
    k = min(r, n - 2)
    S = np.arange(n - k, n)
    assert np.linalg.matrix_rank(G[:, S]) == k
    Y, fac = geninv(G, return_factors=True, keep=_forced_set(n, S))
    assert fac["rank"] == k
    Yx = np.zeros_like(Y)
    Yx[S] = _qr_pinv(G[:, S])
    assert _rel(Y, Yx) < 1e-11, _rel(Y, Yx)
    assert np.all(Y[: n - k] == 0.0)


# columns: g with |g|^2 = 9 (a perfect square, so its repeat's pivot is
# 9 - 3 * 3 = 0 exactly in FP64), g again, another column, a zero column
_REPEATED = [[1, 1, 0, 0], [2, 2, 1, 0], [2, 2, 0, 0], [0, 0, 3, 0], [0, 0, 1, 0]]


def test_forced_pivot_that_is_not_positive_is_rejected():
    """An exactly repeated column and a zero column: their pivots are
    exactly 0, so forcing them kept still rejects them; the result is the
    exact rational pseudoinverse."""
    G = _REPEATED
    Gf = np.array(G, dtype=np.float64)
    Yx = np.array([[float(v) for v in row] for row in exact_pinv(G)])
    Y, fac = geninv(Gf, return_factors=True, keep=np.ones(4, dtype=bool))
    assert fac["rank"] == 2
    assert fac["accepted"].tolist() == [True, False, True, False]
    assert np.max(np.abs(Y - Yx)) <= 1e-12 * np.max(np.abs(Yx))


# --------------------------------------------------------------------------
# planted mistakes in a copy of the forced branch
# --------------------------------------------------------------------------

def _forced_mutant(kind):
    def run(G, keep):
        A = oracle.gram(G)
        n = A.shape[0]
        L = np.zeros((n, n))
        r = 0
        for k in range(n):
            v = A[k:, k] - L[k:, :r] @ L[k, :r]
            kk = min(k + 1, n - 1) if kind == "mask_shift" else k
            take = keep[kk] and (v[0] > 0 or kind == "no_guard")
            if kind == "ignore_keep":
                take = v[0] > pivot_tolerance(A)
            if take:
                d = math.sqrt(v[0]) if v[0] > 0 else 0.0
                L[k, r] = d
                if kind == "fill_from_top":
                    L[:, r] = A[:, k] - L[:, :r] @ L[k, :r]
                    L[:, r] /= d
                    L[k, r] = d
                else:
                    L[k + 1:, r] = v[1:] / d
                r += 1
        L = L[:, :r]
        M = np.linalg.inv(L.T @ L)
        return L @ M @ M @ L.T @ G.T
    return run


def _keep_pins_pass(fn):
    try:
        G = inputs.rank_deficient(45, 20, 11, 5)
        S = np.arange(9, 20)
        Yx = np.zeros((20, 45))
        Yx[S] = _qr_pinv(G[:, S])
        if _rel(fn(G, _forced_set(20, S)), Yx) > 1e-11:
            return False
        G = inputs.full_rank(50, 12, seed=7)
        S = np.sort(np.random.default_rng(7).choice(12, size=7, replace=False))
        if _rel(fn(G, _forced_set(12, S)), _theorem1(_forced_factor(oracle.gram(G), S), G)) > 1e-10:
            return False
        G = _REPEATED
        Yx = np.array([[float(v) for v in row] for row in exact_pinv(G)])
        Y = fn(np.array(G, dtype=np.float64), np.ones(4, dtype=bool))
        if not np.all(np.isfinite(Y)) or np.max(np.abs(Y - Yx)) > 1e-12 * np.max(np.abs(Yx)):
            return False
        return True
    except (np.linalg.LinAlgError, ValueError, FloatingPointError, ZeroDivisionError):
        return False


def test_forced_branch_copy_passes():
    assert _keep_pins_pass(_forced_mutant("none"))


@pytest.mark.parametrize("kind", ["mask_shift", "no_guard", "ignore_keep", "fill_from_top"])
def test_forced_branch_mistakes_are_caught(kind):
    with np.errstate(all="ignore"):
        assert not _keep_pins_pass(_forced_mutant(kind)), kind


def test_oracle_forced_branch_passes_the_same_pins():
    assert _keep_pins_pass(lambda G, keep: geninv(G, keep=keep))
