"""RBF design matrices on the GPU (cpinv_rbf_design) and the normal
equations formed without G in memory (cpinv_rbf_normal_equations) against
the oracle's definition of G (oracle/rbf.py) and its correctly rounded
products (oracle.exact_cross); and W = G+ F through the fused route
against the oracle on an RBF instance with a pivot gap."""
import ctypes

import numpy as np
import pytest

import oracle
import oracle.rbf as orbf
from paper_0804_4809_gb300 import inputs
from tests.gpu_util import TOL, rel, to_dev

pytestmark = pytest.mark.gpu


def _cp():
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _data(m, n, d, seed, on_data=True):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (m, d))
    C = X[np.sort(rng.choice(m, n, replace=False))] if on_data else rng.uniform(-0.2, 1.2, (n, d))
    return X, C


@pytest.mark.parametrize("m,n,d,w,on_data", [(300, 70, 5, 0.3, True), (1000, 130, 8, 0.3, False),
                                             (65, 33, 1, 0.05, False), (130, 40, 32, 0.7, True)])
def test_design_matches_definition(m, n, d, w, on_data):
    cp = _cp()
    X, C = _data(m, n, d, seed=m + n, on_data=on_data)
    G = cp.rbf_design(to_dev(X), to_dev(C), w).cpu().numpy()
    Go = orbf.design(X, C, w)
    # same sum of squares (FMA vs separate rounding: a few ulps of d2) and
    # the same exponential up to its last bits
    big = Go > 1e-300
    assert np.max(np.abs(G[big] - Go[big]) / Go[big]) <= 1e-13
    if (~big).any():
        assert np.max(np.abs(G[~big])) <= 1e-300
    if on_data:
        assert np.sum(G == 1.0) >= n


def test_design_zero_width_and_bad_arguments():
    cp = _cp()
    import torch
    X, C = _data(50, 10, 3, 7)
    with pytest.raises(cp.CpinvError):
        cp.rbf_design(to_dev(X), to_dev(C), 0.0)
    X40, C40 = _data(50, 10, 40, 8)
    with pytest.raises(cp.CpinvError) as e:
        cp.rbf_design(to_dev(X40), to_dev(C40), 0.3)
    assert e.value.status == 6
    # empty shapes are no-ops
    G = cp.rbf_design(torch.zeros((0, 3), dtype=torch.float64, device="cuda:0"), to_dev(C), 0.3)
    assert G.shape == (0, 10)


@pytest.mark.parametrize("m,n,d,k", [(700, 90, 8, 3), (5000, 300, 4, 16), (9000, 64, 8, 1)])
def test_normal_equations_match_oracle_and_materialised_route(m, n, d, k):
    """A = G'G and B = G'F: each chunk of at most 4096 rows exact and
    rounded once (5000 and 9000 rows: two and three chunks).  Against the
    oracle's correctly rounded products of ITS G (the two G differ by a few
    ulps), and against the same products of the GPU's own G materialised
    (cpinv_gram_update, exact-slice), which differ only where the fused
    route's per-centre scale bound sits one binade above the exact one."""
    cp = _cp()
    import torch
    X, C = _data(m, n, d, seed=m, on_data=True)
    F = np.random.default_rng(m + 1).standard_normal((m, k))
    A, B = cp.rbf_normal_equations(to_dev(X), to_dev(C), 0.3, to_dev(F))
    A = A.cpu().numpy()
    B = B.cpu().numpy()
    Go = orbf.design(X, C, 0.3)
    Ao = oracle.exact_cross(Go, Go)
    Bo = oracle.exact_cross(Go, F)
    lo = np.tril_indices(n)
    scale = np.sqrt(np.outer(np.diag(Ao), np.diag(Ao)))[lo]
    assert np.max(np.abs(A[lo] - Ao[lo]) / scale) <= 1e-13
    assert rel(B, Bo) <= 1e-12
    # the materialised route on the GPU's own G
    Gd = cp.rbf_design(to_dev(X), to_dev(C), 0.3)
    Am = torch.zeros((n, n), dtype=torch.float64, device="cuda:0")
    Bm = torch.zeros((n, k), dtype=torch.float64, device="cuda:0")
    cp.gram_update(Am, Gd, Bm, to_dev(F), mode="exact")
    Am = Am.cpu().numpy()
    Bm = Bm.cpu().numpy()
    assert np.max(np.abs(A[lo] - Am[lo]) / scale) <= 4e-16
    # cpinv_gram_update cuts G to 53-bit integers for G'F (62 for G'G), the
    # fused route keeps G's 62-bit planes for both: G rounded at 2^-53 of its
    # column maximum, a few units of 1e-16 in B
    assert rel(B, Bm) <= 4e-15


def test_fused_route_solves_a_gapped_rbf_problem():
    """From (X, C, w, F) to W: the fused normal equations and
    cpinv_lstsq_gram on an RBF design whose centres repeat (every pivot at
    least 10x from tol): rank and W equal the oracle's."""
    cp = _cp()
    G, X, idx = inputs.rbf_repeated_centres(4096, 256, 384, 8, 0.3, seed=21)
    C = X[idx]
    F = inputs.smooth_targets(X, 16, 21)
    Go = orbf.design(X, C, 0.3)
    Wo, fac = oracle.geninv(Go, return_factors=True)
    Wo = Wo @ F
    A, B = cp.rbf_normal_equations(to_dev(X), to_dev(C), 0.3, to_dev(F))
    W, r = cp.lstsq_gram(A, B, mode="exact")
    assert r == fac["rank"] == 256
    Wf = oracle.geninv(Go, exact_gram=False) @ F
    bar = max(TOL["exact"], 8.0 * rel(Wf, Wo))
    err = rel(W.cpu().numpy(), Wo)
    print(f"fused RBF route: rank {r}, rel err vs oracle {err:.3e}, bar {bar:.3e}")
    assert err <= bar


def test_normal_equations_report_nonfinite_input():
    cp = _cp()
    X, C = _data(200, 20, 4, 9)
    X[17, 2] = np.nan
    with pytest.raises(cp.CpinvError) as e:
        cp.rbf_normal_equations(to_dev(X), to_dev(C), 0.3)
    assert e.value.status == 2
    lib = cp.lib()
    assert lib.cpinv_rbf_normal_equations_workspace_size(100, 10, 33, 1) == 0
