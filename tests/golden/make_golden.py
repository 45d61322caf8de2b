"""Writes ``exact_pinv_small.json``: exact rational Moore-Penrose inverses of
small integer matrices, computed by ``oracle.exact`` alone (Fraction
arithmetic, full-rank factorisation route; Sec. 1 definition, Sec. 2 Eq. (4)).

The paper prints no worked numerical example, so every stored value here is
written by this script from the oracle's exact-arithmetic routine; the tests
additionally re-verify each stored G+ against the four Penrose conditions in
exact arithmetic.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact import exact_pinv, exact_rank  # noqa: E402

CASES = {
    # rank 1, 2 x 2: G+ = G' / 25
    "rank1_2x2": [[1, 2], [2, 4]],
    # duplicate columns [g g]
    "dup_cols_3x2": [[1, 1], [2, 2], [2, 2]],
    # zero column in the middle
    "zero_col_3x3": [[1, 0, 2], [0, 0, 1], [3, 0, 1]],
    # rectangular diagonal with a zero
    "rect_diag_4x3": [[2, 0, 0], [0, 0, 0], [0, 0, -4], [0, 0, 0]],
    # wide (m < n), rank 2
    "wide_2x4": [[1, 2, 3, 4], [2, 4, 6, 9]],
    # 6 x 5 of rank 2 (third..fifth columns are combinations of the first two)
    "rank2_6x5": [[1, 0, 2, 1, 3], [0, 1, 1, 2, 1], [1, 1, 3, 3, 4],
                  [2, -1, 3, 0, 5], [1, 2, 4, 5, 5], [0, 3, 3, 6, 3]],
    # 6 x 5 of rank 3: c4 = c1 + c3, c5 = c2 - c3
    "rank3_6x5": [[1, 0, 2, 3, -2], [0, 1, 1, 1, 0], [2, 1, 0, 2, 1],
                  [1, 3, 1, 2, 2], [0, 2, 5, 5, -3], [3, 0, 1, 4, -1]],
    # full column rank 5 x 3
    "full_5x3": [[1, 2, 0], [0, 1, 1], [1, 0, 1], [2, 1, 1], [1, 1, 3]],
    # all zero
    "zero_3x2": [[0, 0], [0, 0], [0, 0]],
}


def main():
    out = {}
    for name, G in CASES.items():
        Y = exact_pinv(G)
        out[name] = {
            "G": G,
            "rank": exact_rank(G),
            "pinv": [[f"{x.numerator}/{x.denominator}" for x in row] for row in Y],
        }
    path = os.path.join(HERE, "exact_pinv_small.json")
    with open(path, "w") as f:
        f.write("{\n")
        items = list(out.items())
        for i, (name, case) in enumerate(items):
            sep = "," if i + 1 < len(items) else ""
            f.write(f" {json.dumps(name)}: {json.dumps(case)}{sep}\n")
        f.write("}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
