"""GPU parity of the normal-equation entry points (incremental learning,
Sec. 4): A += G'G, B += G'F over blocks of rows, then W from A and B, against
the oracle's lstsq on all rows and its lstsq_from_gram on the same A, B."""
import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs

from gpu_util import rel, to_dev, tol_for

pytestmark = pytest.mark.gpu

MODES = ["fp64", "exact"]


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_4809_gb300 import build
    build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _accumulate(cp, G, F, cuts, mode):
    import torch
    n, k = G.shape[1], F.shape[1]
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda:0")
    B = torch.zeros((n, k), dtype=torch.float64, device="cuda:0")
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        cp.gram_update(A, to_dev(G[lo:hi]), B, to_dev(F[lo:hi]), mode=mode)
    torch.cuda.synchronize()
    return A, B


@pytest.mark.parametrize("mode", MODES)
def test_gram_update_matches_gram(cp, mode):
    """One increment from zero: the lower triangle of G'G and G'F (the
    exact-slice Gram agrees with the correctly rounded one to an ulp or so;
    the FP64 one to the summation error m u |G|^2)."""
    G = inputs.normal((333, 70), seed=11)
    F = inputs.normal((333, 4), seed=12)
    A, B = _accumulate(cp, G, F, [0, 333], mode)
    A = A.cpu().numpy()
    Ao = oracle.gram(G)
    low = np.tril_indices(70)
    bar = 4e-16 if mode == "exact" else 333 * 2.0 ** -53
    err = np.abs(A[low] - Ao[low]).max() / np.abs(Ao).max()
    assert err <= bar
    assert not np.triu(A, 1).any()        # the upper triangle is left alone
    assert rel(B.cpu().numpy(), oracle.exact_cross(G, F)) <= bar


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(600, 100, 70, 3), (257, 129, 129, 1), (90, 40, 0, 2),
                                   (1000, 64, 33, 5)])
def test_incremental_matches_lstsq(cp, mode, shape):
    """Rows arrive in ragged blocks (one of a single row); W from the
    accumulated A and B equals lstsq over all rows."""
    m, n, r, k = shape
    G = inputs.rank_deficient(m, n, r, seed=m + 3 * n)
    F = inputs.normal((m, k), seed=k + 5)
    cuts = sorted({0, m, min(m, 128), min(m, 129), min(m, 300), m // 2})
    A, B = _accumulate(cp, G, F, cuts, mode)
    W, rk = cp.lstsq_gram(A, B, mode=mode)
    Wo = oracle.lstsq(G, F)
    assert rk == r
    assert rel(W.cpu().numpy(), Wo) <= 2 * tol_for(mode, G, r)


@pytest.mark.parametrize("mode", MODES)
def test_lstsq_gram_vs_oracle_from_gram(cp, mode):
    """Same A and B on both sides (the oracle's); the strict upper triangle
    of the device copy holds NaN, which the solver must not read."""
    import torch
    G = inputs.rank_deficient(400, 150, 110, seed=21)
    F = inputs.normal((400, 6), seed=22)
    A = oracle.gram(G)
    B = oracle.exact_cross(G, F)
    Wo, ro = oracle.lstsq_from_gram(A, B)
    Ad = A.copy()
    Ad[np.triu_indices(150, 1)] = np.nan
    W, rk = cp.lstsq_gram(to_dev(Ad), to_dev(B), mode=mode)
    torch.cuda.synchronize()
    assert rk == ro == 110
    assert rel(W.cpu().numpy(), Wo) <= tol_for(mode, G, ro)
    # rank only (k = 0)
    _, r0 = cp.lstsq_gram(to_dev(Ad), to_dev(B[:, :0]), mode=mode)
    assert r0 == 110


def test_lstsq_gram_edge_cases(cp):
    import torch
    # n = 0
    W, r = cp.lstsq_gram(torch.zeros((0, 0), dtype=torch.float64, device="cuda:0"),
                         torch.zeros((0, 2), dtype=torch.float64, device="cuda:0"))
    assert r == 0 and W.shape == (0, 2)
    # A = 0: rank 0, W = 0
    W, r = cp.lstsq_gram(torch.zeros((9, 9), dtype=torch.float64, device="cuda:0"),
                         torch.ones((9, 2), dtype=torch.float64, device="cuda:0"))
    torch.cuda.synchronize()
    assert r == 0 and not W.cpu().numpy().any()
    # an empty row block leaves A and B unchanged
    A = torch.eye(5, dtype=torch.float64, device="cuda:0")
    B = torch.ones((5, 1), dtype=torch.float64, device="cuda:0")
    cp.gram_update(A, torch.zeros((0, 5), dtype=torch.float64, device="cuda:0"), B,
                   torch.zeros((0, 1), dtype=torch.float64, device="cuda:0"))
    torch.cuda.synchronize()
    assert torch.equal(A.cpu(), torch.eye(5, dtype=torch.float64))
    assert torch.equal(B.cpu(), torch.ones((5, 1), dtype=torch.float64))
