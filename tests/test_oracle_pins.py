"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* exact rational G+ (fractions, full-rank-factorisation route) on tiny integer
  matrices, stored in tests/golden/ and re-verified here against the four
  Penrose conditions in exact arithmetic (Sec. 1);
* the four Penrose conditions on the benchmark-shaped inputs (Sec. 1, Sec. 3);
* the full-rank closed form (G'G)^-1 G' of Sec. 1, computed by another route
  (Householder QR: G+ = R^-1 Q');
* a hand-written one-sided Jacobi SVD pseudoinverse on tiny inputs (itself
  pinned to LAPACK's SVD);
* special cases with closed forms, and invariances of G+;
* Eq. (1) (G'G = LL') and the structure of S / L of Sec. 2;
* the tolerance rule of the Appendix;
* planted mistakes in copies of the oracle's formulas, each of which must be
  caught by one of these pins.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.exact import exact_pinv, exact_rank
from oracle.geninv import full_rank_cholesky, geninv, pivot_tolerance
from oracle.jacobi import jacobi_svd, jacobi_svd_pinv
from paper_0804_4809_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "exact_pinv_small.json")


def _frac(s):
    a, b = s.split("/")
    return Fraction(int(a), int(b))


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# --------------------------------------------------------------------------
# exact rational golden values
# --------------------------------------------------------------------------

def _exact_penrose_ok(G, Y):
    """The four Penrose conditions, exactly, in Fraction arithmetic."""
    def mm(A, B):
        return [[sum((a * b for a, b in zip(row, col)), Fraction(0)) for col in zip(*B)] for row in A]

    def tr(A):
        return [list(c) for c in zip(*A)]
    G = [[Fraction(x) for x in row] for row in G]
    GY = mm(G, Y)
    YG = mm(Y, G)
    return (mm(GY, G) == G and mm(YG, Y) == Y and tr(GY) == GY and tr(YG) == YG)


def test_golden_exact_values_satisfy_penrose_exactly():
    cases = json.load(open(GOLDEN))
    assert len(cases) >= 8
    for name, c in cases.items():
        Y = [[_frac(s) for s in row] for row in c["pinv"]]
        assert _exact_penrose_ok(c["G"], Y), name
        # and the script's routine still reproduces the stored values
        assert exact_pinv(c["G"]) == Y, name
        assert exact_rank(c["G"]) == c["rank"], name


def test_oracle_matches_exact_golden():
    cases = json.load(open(GOLDEN))
    for name, c in cases.items():
        G = np.array(c["G"], dtype=np.float64)
        Yx = np.array([[float(_frac(s)) for s in row] for row in c["pinv"]])
        Y, fac = geninv(G, return_factors=True)
        assert fac["rank"] == c["rank"], name
        assert np.max(np.abs(Y - Yx)) <= 1e-12 * max(1.0, np.max(np.abs(Yx))), name


@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_exact_random_integer(seed):
    g = np.random.default_rng(1000 + seed)
    m = int(g.integers(2, 7))
    n = int(g.integers(1, 6))
    r = int(g.integers(0, min(m, n) + 1))
    A = g.integers(-3, 4, (m, r))
    B = g.integers(-3, 4, (r, n))
    Gi = (A @ B).astype(int).tolist() if r > 0 else [[0] * n for _ in range(m)]
    Yx = np.array([[float(x) for x in row] for row in exact_pinv(Gi)]).reshape(n, m)
    Y, fac = geninv(np.array(Gi, dtype=np.float64).reshape(m, n), return_factors=True)
    assert fac["rank"] == exact_rank(Gi)
    assert np.max(np.abs(Y - Yx)) <= 1e-11 * max(1.0, np.max(np.abs(Yx)))


# --------------------------------------------------------------------------
# Penrose conditions on the benchmark-shaped families (Sec. 1, Sec. 3)
# --------------------------------------------------------------------------

def _penrose_normwise(G, Y):
    res = oracle.penrose_residuals(G, Y)
    nG = np.linalg.norm(G)
    nY = np.linalg.norm(Y)
    GY = np.linalg.norm(G @ Y)
    YG = np.linalg.norm(Y @ G)
    return max(res["GYG-G:fro"] / nG, res["YGY-Y:fro"] / nY,
               res["sym(GY):fro"] / max(GY, 1e-300), res["sym(YG):fro"] / max(YG, 1e-300))


def test_small_workload_rank_and_penrose():
    G = inputs.workload_small()
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == 80
    # normwise Penrose residuals at the method's FP64 level: u * kappa(T) * kappa(L)
    # with kappa(T) ~ 5e3 for this input (about 1.5e-11); 2e-10 is Sec. 3's figure
    assert _penrose_normwise(G, Y) < 2e-10
    # the wide gap the inputs are built to have: smallest kept pivot far above
    # tol, largest rejected far below it
    piv = fac["pivots"]
    acc = fac["accepted"]
    assert piv[acc].min() > 1e3 * fac["tol"]
    assert np.abs(piv[~acc]).max() < 5e-2 * fac["tol"]


@pytest.mark.parametrize("n", [32, 64, 128])
def test_paper_family_penrose_bound(n):
    """Sec. 3: every coefficient of the four error matrices <= 2e-10 for the
    m = 2n, r = 7n/8, [-1,1] family."""
    G = inputs.paper_family(n, seed=n)
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == 7 * n // 8
    res = oracle.penrose_residuals(G, Y)
    for k, v in res.items():
        if k.endswith(":max"):
            assert v <= 2e-10, (k, v)


def test_wide_branch_is_transpose():
    """Appendix transpose branch (m < n): G+ = ((G')+)'."""
    G = inputs.rank_deficient(30, 70, 12, seed=5)
    Y = geninv(G)
    Yt = geninv(G.T)
    assert Y.shape == (70, 30)
    assert _rel(Y, Yt.T) < 1e-12
    assert _penrose_normwise(G, Y) < 1e-10


# --------------------------------------------------------------------------
# the correctly rounded Gram matrix
# --------------------------------------------------------------------------

def test_exact_gram_matches_fraction_arithmetic():
    """Sampled entries of oracle.gram equal the exact rational dot product
    rounded once (Python Fraction -> float is correctly rounded)."""
    G = inputs.rank_deficient(700, 40, 25, seed=21)
    G[:, 3] *= 1e-7                      # columns of very different scale
    G[5, 7] = 3.0e5                      # one large entry in a column
    A = oracle.gram(G)
    g = np.random.default_rng(22)
    for _ in range(60):
        j, l = (int(x) for x in g.integers(0, 40, 2))
        ex = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(G[:, j], G[:, l])), Fraction(0))
        want = float(ex)
        got = A[j, l]
        assert got == want or abs(got - want) <= np.spacing(abs(want)), (j, l, got, want)


def test_exact_gram_integers_and_blas():
    g = np.random.default_rng(23)
    Gi = g.integers(-1000, 1000, (300, 17)).astype(np.float64)
    assert np.array_equal(oracle.gram(Gi), Gi.T @ Gi)   # small integers: exact either way
    G = inputs.normal((513, 33), seed=24)
    assert _rel(oracle.gram(G), G.T @ G) < 1e-15
    assert np.array_equal(oracle.gram(np.zeros((4, 3))), np.zeros((3, 3)))
    assert oracle.gram(np.zeros((0, 3))).shape == (3, 3)



# --------------------------------------------------------------------------
# Full-rank closed form of Sec. 1, by a different route (Householder QR)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(300, 120), (64, 64), (50, 7)])
def test_full_rank_closed_form_via_qr(shape):
    m, n = shape
    G = inputs.full_rank(m, n, seed=m + n)
    Q, R = np.linalg.qr(G)            # Householder QR (LAPACK dgeqrf)
    Yqr = np.linalg.solve(R, Q.T)     # R^-1 Q'  =  (G'G)^-1 G'
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == n
    assert _rel(Y, Yqr) < 1e-11


# --------------------------------------------------------------------------
# hand-written Jacobi SVD pinv: pinned to LAPACK, then compared with the oracle
# --------------------------------------------------------------------------

def test_jacobi_svd_pinned_to_lapack():
    G = inputs.normal((20, 9), seed=3)
    U, s, V = jacobi_svd(G)
    assert np.allclose(np.sort(s)[::-1], np.linalg.svd(G, compute_uv=False), rtol=1e-12, atol=0)
    assert np.allclose(U @ V.T, G, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(9), atol=1e-12)
    assert _rel(jacobi_svd_pinv(G), np.linalg.pinv(G)) < 1e-12


@pytest.mark.parametrize("m,n,r,seed", [(40, 24, 15, 1), (16, 16, 9, 2), (30, 12, 12, 3),
                                        (12, 30, 7, 4), (64, 48, 40, 5)])
def test_oracle_vs_jacobi_svd_pinv(m, n, r, seed):
    G = inputs.rank_deficient(m, n, r, seed)
    Yj = jacobi_svd_pinv(G, rel_threshold=1e-8)
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == r
    assert _rel(Y, Yj) < 1e-10


# --------------------------------------------------------------------------
# special cases with closed forms, and invariances
# --------------------------------------------------------------------------

def test_zero_matrix():
    Y, fac = geninv(np.zeros((5, 3)), return_factors=True)
    assert fac["rank"] == 0 and fac["tol"] is None
    assert Y.shape == (3, 5) and not Y.any()


def test_empty_shapes():
    for shape in [(0, 0), (0, 4), (4, 0)]:
        Y, fac = geninv(np.zeros(shape), return_factors=True)
        assert Y.shape == shape[::-1] and fac["rank"] == 0


def test_single_column():
    g = inputs.normal((17, 1), seed=9)
    assert _rel(geninv(g), g.T / float(g[:, 0] @ g[:, 0])) < 1e-14


def test_duplicate_columns():
    g = inputs.normal((11, 1), seed=10)
    G = np.hstack([g, g])
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == 1
    expect = np.vstack([g.T, g.T]) / (2.0 * float(g[:, 0] @ g[:, 0]))
    assert _rel(Y, expect) < 1e-13


def test_zero_column_gives_zero_row():
    G = inputs.normal((12, 5), seed=11)
    G[:, 2] = 0.0
    Y = geninv(G)
    assert not Y[2].any()
    keep = [0, 1, 3, 4]
    assert _rel(Y[keep], geninv(G[:, keep])) < 1e-13


def test_orthonormal_columns():
    Q, _ = np.linalg.qr(inputs.normal((20, 6), seed=12))
    assert _rel(geninv(Q), Q.T) < 1e-13


def test_rank_one_outer_product():
    u = inputs.normal((9,), seed=13)
    v = inputs.normal((6,), seed=14)
    G = np.outer(u, v)
    expect = np.outer(v, u) / ((u @ u) * (v @ v))
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == 1
    assert _rel(Y, expect) < 1e-13


def test_rectangular_diagonal():
    G = np.zeros((7, 5))
    d = [3.0, 0.0, -0.5, 2.0, 0.0]
    for i, x in enumerate(d):
        G[i, i] = x
    expect = np.zeros((5, 7))
    for i, x in enumerate(d):
        if x != 0:
            expect[i, i] = 1.0 / x
    assert np.max(np.abs(geninv(G) - expect)) < 1e-15


def test_invariances():
    G = inputs.rank_deficient(25, 14, 9, seed=15)
    Y = geninv(G)
    assert _rel(geninv(Y), G) < 1e-10                 # (G+)+ = G
    assert _rel(geninv(G.T), Y.T) < 1e-12             # (G')+ = (G+)'
    assert _rel(geninv(-3.5 * G), Y / -3.5) < 1e-12   # (cG)+ = G+/c
    g = np.random.default_rng(16)
    P = np.eye(25)[g.permutation(25)]
    Qp = np.eye(14)[:, g.permutation(14)]
    assert _rel(geninv(P @ G @ Qp), Qp.T @ Y @ P.T) < 1e-11


# --------------------------------------------------------------------------
# Eq. (1) and the structure of L (Sec. 2)
# --------------------------------------------------------------------------

def test_factor_structure_eq1():
    G = inputs.rank_deficient(120, 60, 41, seed=17)
    A = G.T @ G
    tol = pivot_tolerance(A)
    L, acc, piv = full_rank_cholesky(A, tol)
    r = L.shape[1]
    assert r == 41 and acc.sum() == r
    assert _rel(L @ L.T, A) < 1e-14 * 60
    kept = np.flatnonzero(acc)
    for j, k in enumerate(kept):
        assert L[k, j] > 0                   # positive pivot
        assert not L[:k, j].any()            # zero above the pivot row (S upper triangular)
    # L restricted to the kept rows is lower triangular, non-singular
    T = L[kept]
    assert np.allclose(T, np.tril(T)) and np.all(np.diag(T) > 0)


def test_tolerance_rule():
    A = np.diag([0.0, 4.0, -1.0, 2.0])
    assert pivot_tolerance(A) == pytest.approx(2e-9, rel=1e-15)
    assert pivot_tolerance(np.diag([0.0, -1.0])) is None
    assert pivot_tolerance(A, rel_tol=1e-3) == pytest.approx(2e-3, rel=1e-15)


def test_tolerance_uses_smallest_positive_diagonal():
    G = np.diag([1.0, 1e-5, 0.0])[:, :2]
    Y, fac = geninv(G, return_factors=True)
    assert fac["rank"] == 2
    assert np.max(np.abs(Y - np.diag([1.0, 1e5, 0.0])[:2, :])) < 1e-9


def test_nan_pivot_is_rejected():
    A = np.array([[1.0, 0.0], [0.0, np.nan]])
    L, acc, _ = full_rank_cholesky(A, 1e-9)
    assert acc.tolist() == [True, False]


def test_listing_literal_reading_agrees_on_exact_rank():
    """The listing's leftover residual (reading of the Appendix) changes G+
    only at the rounding level on inputs of exact rank."""
    G = inputs.workload_small()
    Y0 = geninv(G)
    Y1, fac = geninv(G, literal=True, return_factors=True)
    assert fac["rank"] == 80
    assert _rel(Y1, Y0) < 1e-12


# --------------------------------------------------------------------------
# least squares (Sec. 1)
# --------------------------------------------------------------------------

def test_lstsq_normal_equations_and_min_norm():
    G = inputs.rank_deficient(90, 40, 25, seed=18)
    F = inputs.normal((90, 3), seed=19)
    W = oracle.lstsq(G, F)
    nG = np.linalg.norm(G)
    assert np.linalg.norm(G.T @ (G @ W - F)) < 1e-10 * nG * nG * np.linalg.norm(W)
    Y = geninv(G)
    # W lies in the row space of G:  (I - G+G) W = 0
    assert np.linalg.norm(W - Y @ (G @ W)) < 1e-12 * np.linalg.norm(W)
    # any other LS solution W + z (z in null(G)) has a larger norm
    z = (np.eye(40) - Y @ G) @ inputs.normal((40, 3), seed=20)
    assert np.linalg.norm(G @ z) < 1e-10 * np.linalg.norm(z)
    assert np.linalg.norm(W + z) > np.linalg.norm(W)


# --------------------------------------------------------------------------
# planted mistakes: each mutant of the oracle must fail at least one pin
# --------------------------------------------------------------------------

def _mutant(kind):
    def run(G):
        G = np.asarray(G, dtype=np.float64)
        A = oracle.gram(G)
        dA = np.diag(A)
        pos = dA[dA > 0]
        tol = (pos.max() if kind == "tol_max" else pos.min()) * 1e-9
        n = A.shape[0]
        L = np.zeros((n, n))
        r = 0
        for k in range(n):
            if kind == "drop_update":
                v = A[k:, k].copy()
            elif kind == "sign_update":
                v = A[k:, k] + L[k:, :r] @ L[k, :r]
            elif kind == "index_update":
                v = A[k:, k] - L[k:, :r] @ L[min(k + 1, n - 1), :r]
            else:
                v = A[k:, k] - L[k:, :r] @ L[k, :r]
            thr = 0.0 if kind == "zero_tol" else tol
            if v[0] > thr:
                d = v[0] if kind == "no_sqrt" else math.sqrt(v[0])
                L[k, r] = d
                L[k + 1:, r] = v[1:] / d
                r += 1
        L = L[:, :r]
        M = np.linalg.inv(L.T @ L)
        if kind == "single_M":
            return L @ M @ L.T @ G.T
        if kind == "G_not_transposed":
            return (L @ M @ M @ L.T) @ G.T[:, ::-1]
        return L @ M @ M @ L.T @ G.T
    return run


def _pins_pass(fn):
    """The float pins above, in compact form: returns True iff all hold."""
    try:
        cases = json.load(open(GOLDEN))
        for c in cases.values():
            G = np.array(c["G"], dtype=np.float64)
            if G.shape[0] < G.shape[1] or not G.any():
                continue
            Yx = np.array([[float(_frac(s)) for s in row] for row in c["pinv"]])
            if np.max(np.abs(fn(G) - Yx)) > 1e-12 * max(1.0, np.max(np.abs(Yx))):
                return False
        G = inputs.rank_deficient(40, 24, 15, 1)
        if _rel(fn(G), jacobi_svd_pinv(G)) > 1e-10:
            return False
        G = inputs.workload_small()
        if _penrose_normwise(G, fn(G)) > 2e-10:
            return False
        # tol is 1e-9 times the SMALLEST positive diagonal entry: a column
        # 1e-5 times smaller than another is still kept
        D = np.diag([1.0, 1e-5, 0.0])[:, :2]
        if np.max(np.abs(fn(D) - np.diag([1.0, 1e5, 0.0])[:2, :])) > 1e-9:
            return False
        G = inputs.full_rank(50, 7, seed=57)
        Q, R = np.linalg.qr(G)
        if _rel(fn(G), np.linalg.solve(R, Q.T)) > 1e-11:
            return False
        return True
    except (np.linalg.LinAlgError, ValueError, FloatingPointError, ZeroDivisionError):
        return False


def test_correct_formula_passes_compact_pins():
    assert _pins_pass(_mutant("none"))


@pytest.mark.parametrize("kind", ["drop_update", "sign_update", "index_update", "no_sqrt",
                                  "single_M", "G_not_transposed", "zero_tol", "tol_max"])
def test_planted_mistakes_are_caught(kind):
    with np.errstate(all="ignore"):
        assert not _pins_pass(_mutant(kind)), kind


def test_lstsq_from_gram_matches_lstsq():
    """Theorem 1 applied to F needs G only through A = G'G and B = G'F:
    from the correctly rounded A and B the result equals lstsq(G, F) (the
    two differ only in where G'F is rounded), and the normal equations
    hold."""
    G = inputs.rank_deficient(120, 40, 25, 61)
    F = inputs.normal((120, 3), 62)
    W, r = oracle.lstsq_from_gram(oracle.gram(G), oracle.exact_cross(G, F))
    assert r == 25
    W0 = oracle.lstsq(G, F)
    assert np.linalg.norm(W - W0) <= 1e-11 * np.linalg.norm(W0)
    res = G.T @ (G @ W - F)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(G) ** 2 * np.linalg.norm(W)
    # only the lower triangle of A is read
    A = oracle.gram(G)
    A_up = A + np.triu(np.full_like(A, 7.0), 1)
    W2, _ = oracle.lstsq_from_gram(A_up, oracle.exact_cross(G, F))
    assert np.array_equal(W2, W)
