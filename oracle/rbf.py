"""Gaussian radial-basis design matrix, by its definition (CPU, FP64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU legs of
``bench.py``; the library never imports it and shares no code with it.

Sec. 1 and Sec. 4 of the paper: an RBF network's output weights solve
W = G+ F, G the design matrix of its hidden layer,

    G_ij = exp(-|x_i - c_j|^2 / (2 w^2)),

x_i the inputs (rows of X), c_j the centres (rows of C), w the width.  The
squared distance is the plain sum over coordinates of (x_ik - c_jk)^2, in
coordinate order (no expansion into |x|^2 + |c|^2 - 2 x.c, which cancels for
near points).

Parity status: pinned by ``tests/test_oracle_rbf.py`` (distance zero gives
1, symmetry, a one-dimensional closed form, the expanded form of the input
generator within its cancellation bound).
"""
from __future__ import annotations

import numpy as np


def design(X: np.ndarray, C: np.ndarray, width: float) -> np.ndarray:
    """G (m x n) for inputs X (m x d), centres C (n x d) and width w > 0."""
    X = np.asarray(X, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    m, d = X.shape
    n = C.shape[0]
    if C.shape[1] != d:
        raise ValueError("X and C need the same number of coordinates")
    d2 = np.zeros((m, n))
    for k in range(d):
        t = X[:, k][:, None] - C[:, k][None, :]
        d2 += t * t
    return np.exp(-d2 / (2.0 * width * width))
