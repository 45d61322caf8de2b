"""Pins of the oracle's adjoint of W = G+ F (oracle/adjoint.py), each against
something other than the oracle itself:

* central finite differences of the oracle's forward method (FP64, eps = 1e-6,
  S checked unchanged at +-eps; the tolerance comes from the FD's own
  self-consistency, eps against eps/2), on random directions and single
  entries;
* the Golub-Pereyra derivative of the pseudoinverse on inputs of exact rank
  whose rejected columns all come after the kept ones (there the method's
  derivative and the derivative of G+ coincide);
* the full-rank closed form, G+ from a Householder QR;
* planted mistakes in the adjoint, each caught by one of the above.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import adjoint as adj
from oracle.jacobi import jacobi_svd_pinv
from paper_0804_4809_gb300 import inputs

def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _fd_check(vjp, G, F, dW, dirs, eps=1e-6):
    """Max over directions of |<dG, D> - FD| / (FD error estimate + scale)."""
    S0 = oracle.rank(G)[1]
    _, dG, dF = vjp(G, F, dW)

    def f(Gx, Fx):
        return float(np.sum(dW * oracle.lstsq(Gx, Fx)))

    worst = 0.0
    for D, DF in dirs:
        for e in (eps, eps / 2):
            assert np.array_equal(oracle.rank(G + e * D)[1], S0)
            assert np.array_equal(oracle.rank(G - e * D)[1], S0)
        fd1 = (f(G + eps * D, F + eps * DF) - f(G - eps * D, F - eps * DF)) / (2 * eps)
        fd2 = (f(G + eps / 2 * D, F + eps / 2 * DF) - f(G - eps / 2 * D, F - eps / 2 * DF)) / eps
        an = float(np.sum(dG * D) + np.sum(dF * DF))
        scale = (np.linalg.norm(dG) * np.linalg.norm(D) + np.linalg.norm(dF) * np.linalg.norm(DF))
        err_est = 4.0 * abs(fd1 - fd2) + 1e-7 * scale
        worst = max(worst, abs(an - fd2) / err_est)
    return worst


def _dirs(rng, m, n, k, count, singles=0):
    out = [(rng.standard_normal((m, n)), rng.standard_normal((m, k))) for _ in range(count)]
    for _ in range(singles):
        D = np.zeros((m, n))
        D[rng.integers(m), rng.integers(n)] = 1.0
        out.append((D, np.zeros((m, k))))
    return out


def _early_dependent(seed=1):
    """Rank 7, with a rejected column (col 1 = 2 col 0) before kept ones."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((30, 7)) @ rng.standard_normal((7, 12))
    G[:, 1] = 2.0 * G[:, 0]
    return G, rng.standard_normal((30, 3)), rng.standard_normal((12, 3))


CASES = {
    # name: (G, F, dW)
    "rank_deficient": lambda: (inputs.rank_deficient(30, 12, 7, 21), inputs.normal((30, 3), 22),
                               inputs.normal((12, 3), 23)),
    "early_dependent": _early_dependent,
    "full_rank": lambda: (inputs.full_rank(40, 15, 24), inputs.normal((40, 2), 25),
                          inputs.normal((15, 2), 26)),
    "wide": lambda: (inputs.rank_deficient(12, 30, 8, 27), inputs.normal((12, 3), 28),
                     inputs.normal((30, 3), 29)),
    "square_deficient": lambda: (inputs.rank_deficient(25, 25, 10, 30), inputs.normal((25, 2), 31),
                                 inputs.normal((25, 2), 32)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_matches_finite_differences(name):
    G, F, dW = CASES[name]()
    m, n = G.shape
    rng = np.random.default_rng(sum(map(ord, name)))
    worst = _fd_check(adj.lstsq_vjp, G, F, dW, _dirs(rng, m, n, F.shape[1], 16, 64))
    assert worst <= 1.0, worst


def test_adjoint_equals_golub_pereyra_on_exact_rank():
    """Rejected columns after the kept ones (generic G = A B): the method's
    derivative is the derivative of G+ along constant rank."""
    for (m, n, r, seed) in [(30, 12, 7, 41), (40, 20, 20, 42), (12, 30, 8, 43), (25, 25, 10, 44)]:
        G = inputs.rank_deficient(m, n, r, seed)
        F = inputs.normal((m, 3), seed + 100)
        dW = inputs.normal((n, 3), seed + 200)
        _, dG, _ = adj.lstsq_vjp(G, F, dW)
        gp = adj.golub_pereyra_vjp(G, F, dW, jacobi_svd_pinv(G))
        assert _rel(dG, gp) < 1e-9, (m, n, r, _rel(dG, gp))


def test_adjoint_differs_from_golub_pereyra_with_early_rejected_column():
    """With a rejected column before kept ones the method's function has
    structural zeros that G+ does not: the two derivatives differ (and the
    finite differences side with the method, test above)."""
    G, F, dW = _early_dependent()
    _, dG, _ = adj.lstsq_vjp(G, F, dW)
    gp = adj.golub_pereyra_vjp(G, F, dW, jacobi_svd_pinv(G))
    assert _rel(dG, gp) > 1e-2


def test_adjoint_full_rank_closed_form():
    """Full column rank: W = (G'G)^-1 G'F, dG = -G+' dW W' + (F - G W) dW' G+ G+'
    with G+ = R^-1 Q' from a Householder QR; dF = G+' dW."""
    G = inputs.full_rank(50, 9, 45)
    F = inputs.normal((50, 4), 46)
    dW = inputs.normal((9, 4), 47)
    Q, R = np.linalg.qr(G)
    Gp = np.linalg.solve(R, Q.T)
    W = Gp @ F
    ref = -Gp.T @ dW @ W.T + (F - G @ W) @ dW.T @ Gp @ Gp.T
    W_o, dG, dF = adj.lstsq_vjp(G, F, dW)
    assert _rel(W_o, W) < 1e-12
    assert _rel(dG, ref) < 1e-11
    assert _rel(dF, Gp.T @ dW) < 1e-12


def test_adjoint_zero_matrix():
    G = np.zeros((6, 4))
    W, dG, dF = adj.lstsq_vjp(G, np.ones((6, 2)), np.ones((4, 2)))
    assert not W.any() and not dG.any() and not dF.any()


# --------------------------------------------------------------------------
# planted mistakes in the adjoint
# --------------------------------------------------------------------------

MUTANTS = {
    "no_pattern_mask": ("    Lbar = Lbar * pattern\n", "    pass\n"),
    "no_N_symmetrization": ("    Lbar += L @ (Nbar + Nbar.T)\n", "    Lbar += L @ Nbar\n"),
    "phi_full_diagonal": ("    P[np.diag_indices_from(P)] *= 0.5\n", "    P[np.diag_indices_from(P)] *= 1.0\n"),
    "sign_LbS": ("        LbS = LbS - np.linalg.solve(LS.T, LbD.T @ LD)\n",
                 "        LbS = LbS + np.linalg.solve(LS.T, LbD.T @ LD)\n"),
    "drop_second_Mbar": ("    Mbar += c2bar @ c1.T\n    c1bar", "    c1bar"),
    "drop_F_term": ("    dG = G @ (Abar + Abar.T) + F @ Bbar.T\n", "    dG = G @ (Abar + Abar.T)\n"),
    "Abar_not_symmetrized": ("    dG = G @ (Abar + Abar.T) + F @ Bbar.T\n",
                             "    dG = G @ (2.0 * Abar) + F @ Bbar.T\n"),
}


def _load_mutant(kind):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "adjoint.py")).read()
    old, new = MUTANTS[kind]
    assert src.count(old) >= 1, kind
    src = src.replace(old, new, 1)
    mod = type(os)("oracle._adjoint_mutant")
    mod.__package__ = "oracle"
    exec(compile(src, "adjoint_mutant.py", "exec"), mod.__dict__)
    return mod


def _adj_pins_pass(mod):
    try:
        for name in ("early_dependent", "rank_deficient"):
            G, F, dW = CASES[name]()
            rng = np.random.default_rng(7)
            if _fd_check(mod.lstsq_vjp, G, F, dW, _dirs(rng, *G.shape, F.shape[1], 4)) > 1.0:
                return False
        G = inputs.rank_deficient(30, 12, 7, 41)
        F = inputs.normal((30, 3), 141)
        dW = inputs.normal((12, 3), 241)
        _, dG, _ = mod.lstsq_vjp(G, F, dW)
        if _rel(dG, adj.golub_pereyra_vjp(G, F, dW, jacobi_svd_pinv(G))) > 1e-9:
            return False
        return True
    except (np.linalg.LinAlgError, ValueError, FloatingPointError):
        return False


def test_correct_adjoint_passes_compact_pins():
    assert _adj_pins_pass(adj)


@pytest.mark.parametrize("kind", sorted(MUTANTS))
def test_planted_adjoint_mistakes_are_caught(kind):
    with np.errstate(all="ignore"):
        assert not _adj_pins_pass(_load_mutant(kind)), kind
