"""Hand-written one-sided Jacobi (Hestenes) SVD pseudoinverse, for tiny inputs.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` alone).  It is a second,
independent route to G+ that uses no Cholesky factorisation: by uniqueness of
the Moore-Penrose inverse (Sec. 1, the four Penrose conditions) it must agree
with ``oracle.geninv`` whenever both draw the same rank, i.e. on inputs with a
wide singular-value gap.  The SVD method is the comparison the paper names
(Sec. 1, Sec. 3: Matlab ``pinv``).

Algorithm (Hestenes 1958, one-sided Jacobi): repeatedly rotate column pairs
(p, q) of U = G so that they become orthogonal, accumulating the rotations in
V; at convergence U = [u_1 .. u_n] has orthogonal columns, sigma_j = |u_j| and
G = (U diag(1/sigma)) diag(sigma) V'.  Then G+ = V diag(1/sigma_j) (u_j/sigma_j)'
summed over the sigma_j above ``rel_threshold * sigma_max``.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_svd(G: np.ndarray, sweeps: int = 60, eps: float = 1e-15):
    """Return (U_scaled, sigma, V) with G = U_scaled @ V.T, U_scaled having
    mutually orthogonal columns of norm sigma (not normalised)."""
    U = np.array(G, dtype=np.float64, copy=True)
    m, n = U.shape
    V = np.eye(n)
    for _ in range(sweeps):
        off = 0.0
        for p in range(n - 1):
            for q in range(p + 1, n):
                up = U[:, p]
                uq = U[:, q]
                alpha = float(up @ up)
                beta = float(uq @ uq)
                gamma = float(up @ uq)
                if alpha == 0.0 or beta == 0.0:
                    continue
                c_off = abs(gamma) / math.sqrt(alpha * beta)
                off = max(off, c_off)
                if c_off < eps:
                    continue
                # Rotation angle that zeroes the (p, q) entry of U'U.
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                new_p = c * up - s * uq
                new_q = s * up + c * uq
                U[:, p] = new_p
                U[:, q] = new_q
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if off < eps:
            break
    sigma = np.sqrt(np.sum(U * U, axis=0))
    return U, sigma, V


def jacobi_svd_pinv(G: np.ndarray, rel_threshold: float = 1e-8) -> np.ndarray:
    """G+ from the one-sided Jacobi SVD, keeping sigma > rel_threshold*sigma_max."""
    G = np.asarray(G, dtype=np.float64)
    m, n = G.shape
    if m == 0 or n == 0:
        return np.zeros((n, m))
    if m < n:
        return jacobi_svd_pinv(G.T, rel_threshold).T
    U, sigma, V = jacobi_svd(G)
    smax = float(sigma.max()) if sigma.size else 0.0
    Y = np.zeros((n, m))
    if smax == 0.0:
        return Y
    for j in range(n):
        if sigma[j] > rel_threshold * smax:
            u = U[:, j] / sigma[j]
            Y += np.outer(V[:, j] / sigma[j], u)
    return Y
