"""Pivot-gap check of the batched workload, with the oracle only.

A rank-deficient instance G = A B (inner dimension r) has rank r in exact
arithmetic, but the Appendix rank decision compares every pivot with
tol = rel_tol * min positive diagonal entry.  When the kept columns are close
to dependent, a pivot that is zero in exact arithmetic can come out above tol
(or a genuine one below it) by rounding alone, and two correct FP64
evaluations may then disagree on the rank.  Such an instance is re-drawn: it
passes when the oracle's smallest kept pivot is at least 1e3 * tol and its
largest rejected pivot at most 1e-3 * tol.

Run as a script to (re)write ``batched_gap.json``: for the 512-problem batch
workload (seed 4, k = 4), the draw used for each problem slot that needed a
re-draw.  ``bench.py`` and the tests read that file; the test suite checks it
against ``attempts_for`` on the same arguments.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0804_4809_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "batched_gap.json")
WORKLOAD = {"P": 512, "seed": 4, "k": 4, "m_range": [64, 1024], "n_lo": 32, "n_hi": 512}
LO, HI = 1e3, 1e-3


def gap_ok(G: np.ndarray) -> bool:
    """True when every oracle pivot is far from the tolerance."""
    _, f = oracle.geninv(G, return_factors=True)
    piv = np.asarray(f["pivots"], dtype=np.float64)
    acc = np.asarray(f["accepted"]).astype(bool)
    tol = f["tol"]
    if tol is None:
        return True
    if acc.any() and piv[acc].min() < LO * tol:
        return False
    if (~acc).any() and piv[~acc].max() > HI * tol:
        return False
    return True


def attempts_for(P, seed, k=4, m_range=(64, 1024), n_lo=32, n_hi=512, slots=None,
                 max_draws=20) -> dict:
    """{slot: draw} for the slots whose first draw fails the gap check."""
    out = {}
    for i in (range(P) if slots is None else slots):
        for a in range(max_draws):
            p = inputs.batched_problem(seed, i, a, k, m_range, n_lo, n_hi)
            if gap_ok(p.G):
                if a:
                    out[i] = a
                break
        else:
            raise RuntimeError(f"slot {i}: no draw passes the gap check")
    return out


def load() -> dict:
    """The stored draws of the batch workload, as {slot: draw}."""
    with open(OUT) as fh:
        d = json.load(fh)
    return {int(i): int(a) for i, a in d["attempts"].items()}


def main():
    w = WORKLOAD
    att = attempts_for(w["P"], w["seed"], w["k"], tuple(w["m_range"]), w["n_lo"], w["n_hi"])
    doc = {"source": "tests/golden/make_batched_gap.py (oracle pivots; gap 1e3 / 1e-3 x tol)",
           "workload": w, "attempts": {str(i): a for i, a in sorted(att.items())}}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1)
        fh.write("\n")
    print(f"{len(att)} of {w['P']} slots re-drawn -> {OUT}")


if __name__ == "__main__":
    main()
