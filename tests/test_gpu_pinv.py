"""GPU parity of pinv / lstsq / rank against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs

from gpu_util import TOL, dev, penrose_normwise, rel, to_dev, tol_for

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


def _pinv(cp, G, mode, **kw):
    import torch
    Y, r = cp.pinv(to_dev(G), mode=mode, **kw)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), r


@pytest.mark.parametrize("mode", MODES)
def test_small_workload(cp, mode):
    """200 x 100, rank 80: rank, kept mask, G+ and the four Penrose conditions."""
    G = inputs.workload_small()
    Yo, fac = oracle.geninv(G, return_factors=True)
    Y, r = _pinv(cp, G, mode)
    assert r == fac["rank"] == 80
    rk, mask = cp.rank(to_dev(G), mode=mode)
    assert rk == 80
    assert np.array_equal(mask.cpu().numpy().astype(bool), fac["accepted"])
    assert rel(Y, Yo) <= TOL[mode]
    assert penrose_normwise(G, Y) < 1e-9


SHAPES = [
    (200, 100, 80), (130, 70, 70), (64, 200, 31), (1, 1, 1), (17, 1, 1), (1, 17, 1),
    (300, 257, 100), (500, 129, 128), (40, 40, 40), (333, 65, 64), (90, 33, 0),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("panel", [8, 16, 32])
@pytest.mark.parametrize("shape", SHAPES)
def test_shapes_and_panels(cp, mode, panel, shape):
    m, n, r = shape
    G = inputs.rank_deficient(m, n, r, seed=m * 7 + n)
    Yo, fac = oracle.geninv(G, return_factors=True)
    Y, rk = _pinv(cp, G, mode, panel=panel)
    assert rk == fac["rank"] == r
    assert Y.shape == (n, m)
    if r == 0:
        assert not Y.any()
    else:
        assert rel(Y, Yo) <= tol_for(mode, G, r)


@pytest.mark.parametrize("mode", MODES)
def test_lstsq(cp, mode):
    import torch
    for (m, n, r, k) in [(200, 100, 80, 3), (64, 150, 40, 5), (257, 129, 129, 1)]:
        G = inputs.rank_deficient(m, n, r, seed=m + n + k)
        F = inputs.normal((m, k), seed=k)
        Wo = oracle.lstsq(G, F)
        W, rk = cp.lstsq(to_dev(G), to_dev(F), mode=mode)
        torch.cuda.synchronize()
        assert rk == r
        assert rel(W.cpu().numpy(), Wo) <= tol_for(mode, G, r)


@pytest.mark.parametrize("mode", MODES)
def test_special_cases(cp, mode):
    # zero column -> zero row of G+
    G = inputs.normal((50, 9), seed=3)
    G[:, 4] = 0.0
    Y, r = _pinv(cp, G, mode)
    assert r == 8 and not Y[4].any()
    # duplicate columns
    g = inputs.normal((31, 1), seed=4)
    Y, r = _pinv(cp, np.hstack([g, g, g]), mode)
    assert r == 1
    assert rel(Y, np.vstack([g.T] * 3) / (3 * float(g[:, 0] @ g[:, 0]))) < 1e-14
    # G = 0
    Y, r = _pinv(cp, np.zeros((12, 7)), mode)
    assert r == 0 and not Y.any()
    # rectangular diagonal
    G = np.zeros((9, 6))
    for i, x in enumerate([2.0, 0.0, -4.0, 0.5, 0.0, 8.0]):
        G[i, i] = x
    Y, r = _pinv(cp, G, mode)
    assert r == 4
    assert np.max(np.abs(Y - oracle.geninv(G))) < 1e-15


@pytest.mark.parametrize("mode", MODES)
def test_leading_dimensions_and_stream(cp, mode):
    import torch
    m, n, r = 150, 70, 50
    G = inputs.rank_deficient(m, n, r, seed=9)
    big = torch.zeros((m, n + 13), dtype=torch.float64, device=dev())
    big[:, 5:5 + n] = to_dev(G)
    view = big[:, 5:5 + n]            # ldg = n + 13
    outbig = torch.full((n, m + 7), 7.0, dtype=torch.float64, device=dev())
    out = outbig[:, :m]               # ldgp = m + 7
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Y, rk = cp.pinv(view, mode=mode, out=out)
    s.synchronize()
    assert rk == r
    assert rel(out.cpu().numpy(), oracle.geninv(G)) <= tol_for(mode, G, r)
    assert torch.all(outbig[:, m:] == 7.0)   # nothing written past the row length


@pytest.mark.parametrize("mode", MODES)
def test_nonfinite_input_is_reported(cp, mode):
    G = inputs.normal((40, 10), seed=5)
    G[7, 3] = np.nan
    with pytest.raises(cp.CpinvError) as e:
        _pinv(cp, G, mode)
    assert e.value.status == 2
    G[7, 3] = np.inf
    with pytest.raises(cp.CpinvError):
        _pinv(cp, G, mode)


@pytest.mark.parametrize("mode", MODES)
def test_deterministic(cp, mode):
    G = inputs.rank_deficient(300, 200, 150, seed=12)
    Y1, _ = _pinv(cp, G, mode)
    Y2, _ = _pinv(cp, G, mode)
    assert np.array_equal(Y1, Y2)


@pytest.mark.parametrize("mode", MODES)
def test_large_rank_deficient_full_size(cp, mode):
    """4096 x 2048, rank 1536 -- the benchmark workload, element by element."""
    G = inputs.workload_large_rank_deficient()
    Yo, fac = oracle.geninv(G, return_factors=True)
    Y, r = _pinv(cp, G, mode)
    assert r == fac["rank"] == 1536
    e = rel(Y, Yo)
    print(f"4096x2048 r=1536 {mode}: rel err {e:.3e}")
    assert e <= TOL[mode]


@pytest.mark.parametrize("mode", MODES)
def test_large_full_rank_full_size(cp, mode):
    G = inputs.workload_large_full_rank()
    Yo, fac = oracle.geninv(G, return_factors=True)
    Y, r = _pinv(cp, G, mode)
    assert r == fac["rank"] == 2048
    e = rel(Y, Yo)
    print(f"4096x2048 full rank {mode}: rel err {e:.3e}")
    assert e <= TOL[mode]


@pytest.mark.parametrize("mode", MODES)
def test_graph_replay_matches_direct_run(cp, mode):
    """Repeated calls with the same arguments: the first runs the kernels
    directly, the second is captured into a CUDA graph, later ones replay it.
    All must give the same bits, rank and status."""
    import torch
    G = inputs.rank_deficient(700, 300, 210, seed=44)
    Gd = to_dev(G)
    plan = cp.PinvPlan(700, 300, dev(), mode=mode)
    outs = []
    for it in range(4):
        out = torch.empty((300, 700), dtype=torch.float64, device=dev()) if it == 0 else outs[0][1]
        r = plan(Gd, out, sync_rank=True)
        assert r == 210
        outs.append((out.cpu().numpy().copy(), out))
    for Y, _ in outs[1:]:
        assert np.array_equal(Y, outs[0][0])
    assert rel(outs[0][0], oracle.geninv(G)) <= tol_for(mode, G, 210)
    # a replay still reports device-side errors
    Gbad = G.copy()
    Gbad[3, 3] = np.nan
    Gd.copy_(torch.from_numpy(Gbad))
    with pytest.raises(cp.CpinvError) as e:
        plan(Gd, outs[0][1], sync_rank=True)
    assert e.value.status == 2


def test_split_mode_reduced_accuracy_tier(cp):
    """BF16x3 split precision in the Gram and chain products: a reduced-
    accuracy tier.  On a well-conditioned full-rank input it returns the rank
    and an approximate G+; its error is reported against the oracle, not held
    to the FP64 bar."""
    import torch
    G = inputs.full_rank(400, 150, seed=77)
    Yo = oracle.geninv(G)
    Y, r = _pinv(cp, G, "bf16x3")
    assert r == 150
    e = rel(Y, Yo)
    print(f"bf16x3 400x150 full rank: rel err {e:.3e}")
    assert 1e-12 < e < 1e-3
    F = inputs.normal((400, 4), seed=78)
    W, rk = cp.lstsq(to_dev(G), to_dev(F), mode="bf16x3")
    torch.cuda.synchronize()
    assert rk == 150 and rel(W.cpu().numpy(), oracle.lstsq(G, F)) < 1e-3


# Orders and ranks around the triangular inverse's levels: in the exact mode
# the levels of order 512 and 1024 here are block-diagonal residue products
# whose node rows are clipped by the rank on the device -- a node with six
# rows (r = 1030 of 1100), a node with none (r = 1000), ragged last nodes
# (r = 1200 and r = 650).  The kept columns of these inputs are much worse
# conditioned than G itself (kappa(G_S) up to 7e4 against kappa(G) ~ 100),
# and the method amplifies the Gram's rounding through them (Sec. 2): the
# bar is widened to 8x the oracle's own change between a correctly rounded
# and an FP64 Gram, as for the paper family.  A clipping mistake would move
# G+ by O(1).
LEVEL_SHAPES = [(1400, 1100, 1030), (1400, 1100, 1000), (1300, 1200, 1200), (900, 700, 650)]


@pytest.mark.parametrize("shape", LEVEL_SHAPES)
def test_triangular_inverse_levels_exact(cp, shape):
    m, n, r = shape
    G = inputs.rank_deficient(m, n, r, seed=m + 3 * n + r)
    Yo, fac = oracle.geninv(G, return_factors=True)
    sens = rel(oracle.geninv(G, exact_gram=False), Yo)
    Y, rk = _pinv(cp, G, "exact")
    assert rk == fac["rank"] == r
    assert rel(Y, Yo) <= max(tol_for("exact", G, r), 8.0 * sens), (rel(Y, Yo), sens)
