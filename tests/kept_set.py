"""Kept-set gate for inputs without a rank gap (RBF design matrices).

Two correct FP64-class evaluations of the method may disagree on a pivot
that lies within rounding of the tolerance, and once one decision differs
the later pivots are computed for another kept set.  The gate therefore
asks the oracle for the pivots of the GPU's own kept set S (its forced
branch, pinned in test_oracle_keep.py) and accepts S when every decision in
it agrees with the Appendix test (pivot > tol) on those pivots, except at
pivots within a factor ``band`` of tol, where rounding may decide either
way."""
import numpy as np

import oracle


def gate(G, keep, band=10.0, exact_gram=True):
    """Checks the GPU's kept set ``keep`` against the oracle's pivots for it.

    Returns (Y, fac, info): the oracle's G+ and factors for S = keep, and a
    dict with the number of decisions that differ from the oracle's test
    ('disagree'), how many pivots lie within the band ('in_band') and the
    largest factor by which a differing pivot lies from tol ('worst')."""
    keep = np.asarray(keep, dtype=bool)
    Y, fac = oracle.geninv(G, return_factors=True, exact_gram=exact_gram, keep=keep)
    # the forced branch keeps exactly S (a forced pivot that is not positive
    # would be dropped, and then the comparison would not be for S)
    assert np.array_equal(fac["accepted"], keep), "GPU kept a non-positive pivot"
    piv, tol = fac["pivots"], fac["tol"]
    if tol is None:
        assert not keep.any()
        return Y, fac, {"disagree": 0, "in_band": 0, "worst": 1.0}
    test = piv > tol
    near = (piv >= tol / band) & (piv <= tol * band)
    diff = test != keep
    bad = np.flatnonzero(diff & ~near)
    assert bad.size == 0, (
        f"kept-set decisions differ from the oracle's test away from tol at {bad[:8].tolist()} "
        f"(pivot / tol = {(piv[bad[:8]] / tol).tolist()})")
    ratio = np.where(piv > 0, piv / tol, np.inf)
    worst = float(np.max(np.maximum(ratio[diff], 1.0 / ratio[diff]))) if diff.any() else 1.0
    return Y, fac, {"disagree": int(diff.sum()), "in_band": int(near.sum()), "worst": worst}
