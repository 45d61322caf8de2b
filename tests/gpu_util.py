"""Helpers shared by the GPU test modules (no oracle arithmetic here)."""
import numpy as np
import torch

#: Relative Frobenius tolerance of G+ against the oracle, per arithmetic.
#: exact-slice: FP64-accurate products and a Gram rounded like the oracle's,
#: so the only differences are rounding orders in the Cholesky, the inverse and
#: the chain -- measured below 7e-11 on the benchmark inputs; the stated bar is
#: 1e-10.
#: plain FP64: the Gram is summed with FP64 FMAs in the kernel's own order; on
#: rank-deficient Gaussian products the method amplifies a Gram rounding
#: difference of u |G|^2 by about kappa(T) kappa(L) (T = kept block of the
#: factor), which moves G+ by 0.9e-10 .. 2.1e-10 on the 200 x 100 and
#: 4096 x 2048 inputs (measured between two CPU summation orders), so the plain
#: FP64 form is held to 1e-9.
TOL = {"exact": 1e-10, "fp64": 1e-9}

U = 2.0 ** -53


def tol_for(mode, G, rank=None):
    """The stated bar, widened where the input itself is ill-conditioned.

    The method solves through G'G, so a rounding of relative size u anywhere
    before the inverse moves G+ by about u kappa(G)^2 (kappa over the non-zero
    singular values); two correct FP64-class evaluations of the method differ
    by up to a small multiple of that (measured: 0.13 .. 1.1 u kappa^2 on the
    test inputs).  Inputs with kappa(G) below ~1e3 (the benchmark input:
    kappa ~ 60) keep the stated bar."""
    s = np.linalg.svd(np.asarray(G, dtype=np.float64), compute_uv=False)
    if rank is None:
        rank = int(np.sum(s > s[0] * 1e-8)) if s.size and s[0] > 0 else 0
    if rank == 0:
        return TOL[mode]
    kappa = s[0] / s[rank - 1]
    return max(TOL[mode], 8.0 * U * kappa * kappa)


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def dev():
    return torch.device("cuda:0")


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def penrose_normwise(G, Y):
    GY = G @ Y
    YG = Y @ G
    out = []
    nG, nY = np.linalg.norm(G), np.linalg.norm(Y)
    out.append(np.linalg.norm(GY @ G - G) / max(nG, 1e-300))
    out.append(np.linalg.norm(Y @ GY - Y) / max(nY, 1e-300))
    out.append(np.linalg.norm(GY - GY.T) / max(np.linalg.norm(GY), 1e-300))
    out.append(np.linalg.norm(YG - YG.T) / max(np.linalg.norm(YG), 1e-300))
    return float(max(out))
