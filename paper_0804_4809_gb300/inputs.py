"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws matrices.  Both
the CUDA path (through the tests and ``bench.py``) and the CPU oracle consume
its output, so the two always see the same bytes.

Workload families:

* ``rank_deficient``: G = A B with A (m x r) and B (r x n) i.i.d. N(0,1) (or
  U[-1,1]) factors, so G has rank r (up to the rounding of the product) with a
  singular-value gap of about 1e13 between sigma_r and sigma_{r+1}.
* ``paper_family``: the shape of Sec. 3 / Table 1 -- m = 2n, r = 7n/8,
  coefficients in [-1, 1].  How the paper built rank r is not stated; here it
  is the product of two U[-1,1] factors.
* ``rbf_design``: Gaussian radial-basis design matrices G_ij =
  exp(-|x_i - c_j|^2 / (2 w^2)) with inputs uniform in [0,1]^d and centres drawn
  without replacement from the inputs (Sec. 1 and Sec. 4: RBF networks).
* ``smooth_targets``: sums of sinusoids of the inputs plus N(0, sigma) noise.
* ``batched_problems``: many rank-deficient problems of uneven m, n, rank.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def rank_deficient(m: int, n: int, r: int, seed: int, dist: str = "normal") -> np.ndarray:
    """G = A @ B, A m x r, B r x n, FP64, C-contiguous (row-major)."""
    g = _rng(seed)
    if dist == "normal":
        A = g.standard_normal((m, r))
        B = g.standard_normal((r, n))
    elif dist == "uniform":
        A = g.uniform(-1.0, 1.0, (m, r))
        B = g.uniform(-1.0, 1.0, (r, n))
    else:
        raise ValueError(dist)
    if r == 0:
        return np.zeros((m, n))
    return np.ascontiguousarray(A @ B)


def full_rank(m: int, n: int, seed: int) -> np.ndarray:
    """G with i.i.d. N(0,1) entries (full rank min(m, n) almost surely)."""
    return _rng(seed).standard_normal((m, n))


def paper_family(n: int, seed: int) -> np.ndarray:
    """Sec. 3 test family: m = 2n, r = 7n/8, entries from U[-1,1] factors."""
    return rank_deficient(2 * n, n, (7 * n) // 8, seed, dist="uniform")


def rbf_from_centres(X: np.ndarray, C: np.ndarray, width: float) -> np.ndarray:
    """G_ij = exp(-|x_i - c_j|^2 / (2 w^2)), squared distances expanded as
    |x|^2 + |c|^2 - 2 x.c and clamped at 0."""
    d2 = (np.sum(X * X, axis=1)[:, None] + np.sum(C * C, axis=1)[None, :]
          - 2.0 * (X @ C.T))
    np.maximum(d2, 0.0, out=d2)
    return np.ascontiguousarray(np.exp(-d2 / (2.0 * width * width)))


def rbf_design(m: int, n: int, d: int, width: float, seed: int):
    """Gaussian RBF design matrix.  Returns (G, X, centre_index)."""
    g = _rng(seed)
    X = g.uniform(0.0, 1.0, (m, d))
    idx = np.sort(g.choice(m, size=n, replace=False))
    return rbf_from_centres(X, X[idx], width), X, idx


def rbf_repeated_centres(m: int, n_distinct: int, n: int, d: int, width: float, seed: int):
    """RBF design whose n centres repeat n_distinct distinct inputs (the
    extra n - n_distinct columns are copies of earlier or later ones, in a
    shuffled order).  A repeated centre gives an exactly repeated column, so
    the rank is n_distinct with a wide pivot gap: every pivot is either of
    the order of the data or at rounding level.  Returns (G, X, centre_index)."""
    g = _rng(seed)
    X = g.uniform(0.0, 1.0, (m, d))
    base = np.sort(g.choice(m, size=n_distinct, replace=False))
    idx = np.concatenate([base, g.choice(base, size=n - n_distinct, replace=True)])
    g.shuffle(idx)
    return rbf_from_centres(X, X[idx], width), X, idx


def smooth_targets(X: np.ndarray, k: int, seed: int, noise: float = 1e-3) -> np.ndarray:
    """F[:, t] = sin(2 pi omega_t . x + phi_t) + N(0, noise^2) noise."""
    g = _rng(seed + 7919)
    m, d = X.shape
    omega = g.uniform(0.0, 2.0, (k, d))
    phi = g.uniform(0.0, 2.0 * np.pi, k)
    F = np.sin(2.0 * np.pi * (X @ omega.T) + phi[None, :])
    F += noise * g.standard_normal((m, k))
    return np.ascontiguousarray(F)


def normal(shape, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(shape)


@dataclass
class Problem:
    m: int
    n: int
    r: int
    G: np.ndarray
    F: np.ndarray


def _rng_key(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in keys])))


def batched_problem(seed: int, i: int, attempt: int = 0, k: int = 4, m_range=(64, 1024),
                    n_lo: int = 32, n_hi: int = 512) -> "Problem":
    """Problem slot i, draw ``attempt``, of ``batched_problems``: its own
    stream keyed (seed, i, attempt); m ~ U{m_lo..m_hi}, n ~ U{n_lo..min(m,
    n_hi)}, r ~ U{ceil(n/2)..n}, G = A(m x r) B(r x n) with N(0,1) factors,
    F m x k N(0,1)."""
    g = _rng_key(seed, i, attempt)
    m = int(g.integers(m_range[0], m_range[1] + 1))
    n = int(g.integers(n_lo, min(m, n_hi) + 1))
    r = int(g.integers((n + 1) // 2, n + 1))
    A = g.standard_normal((m, r))
    B = g.standard_normal((r, n))
    F = g.standard_normal((m, k))
    return Problem(m, n, r, np.ascontiguousarray(A @ B), F)


def batched_problems(P: int, seed: int, k: int = 4, m_range=(64, 1024),
                     n_lo: int = 32, n_hi: int = 512, attempts: dict | None = None):
    """P rank-deficient least-squares problems of uneven size (``batched_problem``
    for slots 0..P-1).  ``attempts`` maps a slot to the draw to use (default
    0): a re-drawn instance replaces one whose rank decision is too close to
    the tolerance (the pivot-gap check is made by the test suite, which
    stores the draws it chose)."""
    attempts = attempts or {}
    return [batched_problem(seed, i, attempts.get(i, 0), k, m_range, n_lo, n_hi)
            for i in range(P)]


# ---------------------------------------------------------------------------
# Named workloads (sizes of the benchmark configurations).
# ---------------------------------------------------------------------------

def workload_small(seed: int = 0) -> np.ndarray:
    """200 x 100, rank 80 (N(0,1) factors 200x80 and 80x100)."""
    return rank_deficient(200, 100, 80, seed)


def workload_large_rank_deficient(seed: int = 1) -> np.ndarray:
    """4096 x 2048, rank 1536 (N(0,1) factors 4096x1536 and 1536x2048)."""
    return rank_deficient(4096, 2048, 1536, seed)


def workload_large_full_rank(seed: int = 2) -> np.ndarray:
    """4096 x 2048 N(0,1), full rank 2048."""
    return full_rank(4096, 2048, seed)


def workload_rbf(m: int = 16384, n: int = 2048, d: int = 8, k: int = 16,
                 width: float = 0.3, seed: int = 3):
    """RBF least squares: G m x n, F m x k."""
    G, X, _ = rbf_design(m, n, d, width, seed)
    F = smooth_targets(X, k, seed)
    return G, F
