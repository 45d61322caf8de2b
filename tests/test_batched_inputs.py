"""The batched workload's stored re-draws (tests/golden/batched_gap.json)
against the oracle's pivot-gap check, and the rank the construction fixes."""
import numpy as np

import oracle
from paper_0804_4809_gb300 import inputs
from tests.golden import make_batched_gap as gap


def test_stored_draws_pass_the_gap_check_and_fix_the_rank():
    w = gap.WORKLOAD
    att = gap.load()
    assert att, "the workload needs some re-draws"
    for i in range(w["P"]):
        a = att.get(i, 0)
        # every earlier draw of a re-drawn slot fails the check
        for a0 in range(a):
            p0 = inputs.batched_problem(w["seed"], i, a0, w["k"], tuple(w["m_range"]), w["n_lo"],
                                        w["n_hi"])
            assert not gap.gap_ok(p0.G), (i, a0)
        p = inputs.batched_problem(w["seed"], i, a, w["k"], tuple(w["m_range"]), w["n_lo"],
                                   w["n_hi"])
        _, f = oracle.geninv(p.G, return_factors=True)
        piv = np.asarray(f["pivots"])
        acc = np.asarray(f["accepted"]).astype(bool)
        assert f["rank"] == p.r, (i, f["rank"], p.r)
        assert piv[acc].min() >= gap.LO * f["tol"], i
        if (~acc).any():
            assert piv[~acc].max() <= gap.HI * f["tol"], i


def test_gap_check_rejects_near_dependent_instances():
    """Column 2 of G = column 0 + column 1 + a perturbation of relative size
    eps: its pivot is about eps^2 x its diagonal entry.  eps = 1e-5 gives a
    rejected pivot near 0.1 x tol (above 1e-3 x tol); eps = 3e-4 a kept pivot
    near 1e2 x tol (below 1e3 x tol); eps = 1e-2 and 1e-9 are far from tol."""
    rng = np.random.default_rng(5)
    base = rng.standard_normal((40, 6))
    noise = rng.standard_normal(40) * np.linalg.norm(base[:, 0] + base[:, 1]) / np.sqrt(40)

    def with_eps(eps):
        G = base.copy()
        G[:, 2] = G[:, 0] + G[:, 1] + eps * noise
        return G

    assert not gap.gap_ok(with_eps(1e-5))
    assert not gap.gap_ok(with_eps(3e-4))
    assert gap.gap_ok(with_eps(1e-2))
    assert gap.gap_ok(with_eps(1e-9))
