"""Batched least squares (cpinv_lstsq_batched) against the oracle, per problem.

Every problem of a batch is an independent W = G+ F of the Appendix method
with its own tolerance and rank; the batch must give each the same rank as the
oracle and values within the FP64 bar (widened by tol_for on ill-conditioned
problems)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_0804_4809_gb300 import inputs
from tests.golden import make_batched_gap as gap
from tests.gpu_util import TOL, rel, tol_for, to_dev

pytestmark = pytest.mark.gpu


def _cp():
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _problems(P, seed, **kw):
    """Gap-checked batch (slots re-drawn as the oracle's pivot check asks)."""
    att = gap.attempts_for(P, seed, **kw)
    return inputs.batched_problems(P, seed, attempts=att, **kw)


def fp64_bar(G, F, r):
    """The FP64 bar of one problem: the stated 1e-9 (tol_for), or 8 x the
    oracle's own change when its Gram matrix is rounded in FP64 instead of
    correctly, whichever is larger.  The batch sums G'G with FP64 FMAs, so its
    W differs from the oracle's by about that change (a problem whose kept
    columns are close to dependent amplifies the Gram rounding beyond what
    kappa(G) alone predicts: measured up to 2e-8 on the 512-problem batch)."""
    W_x = O.lstsq(G, F)
    W_f = O.lstsq(G, F, exact_gram=False)
    return max(tol_for("fp64", G, r), 8.0 * rel(W_f, W_x))


def _check_against_oracle(probs, Ws, ranks, statuses, idx=None):
    idx = range(len(probs)) if idx is None else idx
    for i in idx:
        p = probs[i]
        assert statuses[i] == 0, (i, statuses[i])
        r_o, _ = O.rank(p.G)
        assert ranks[i] == r_o, (i, ranks[i], r_o)
        W_o = O.lstsq(p.G, p.F)
        W = Ws[i].cpu().numpy()
        assert rel(W, W_o) <= fp64_bar(p.G, p.F, r_o), (i, p.m, p.n, r_o, rel(W, W_o))


def test_batched_small_uneven():
    """24 problems, m in [16, 300], n in [4, min(m, 160)]: spans several n
    buckets, ragged panels and every rank from n/2 to n."""
    probs = _problems(24, 11, k=3, m_range=(16, 300), n_lo=4, n_hi=160)
    cp = _cp()
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs])
    _check_against_oracle(probs, Ws, ranks, st)
    for p, r in zip(probs, ranks):
        assert r == p.r  # gap-checked construction: rank is the inner dimension


@pytest.mark.parametrize("panel", [16, 32])
def test_batched_panels(panel):
    probs = _problems(10, 12, k=2, m_range=(40, 200), n_lo=20, n_hi=140)
    cp = _cp()
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     panel=panel)
    _check_against_oracle(probs, Ws, ranks, st)


def test_batched_graph_replay_identical():
    """Calls 1 (direct + tuning), 2 (captured) and 3 (replayed) agree bit for bit."""
    probs = _problems(12, 13, k=4, m_range=(64, 400), n_lo=32, n_hi=256)
    cp = _cp()
    plan = cp.BatchedLstsq([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs])
    outs = []
    for _ in range(3):
        Ws, ranks, st = plan()
        outs.append(([W.clone() for W in Ws], list(ranks), list(st)))
    for o in outs[1:]:
        assert o[1] == outs[0][1] and o[2] == outs[0][2]
        for a, b in zip(o[0], outs[0][0]):
            assert torch.equal(a, b)
    _check_against_oracle(probs, outs[0][0], outs[0][1], outs[0][2])


def test_batched_matches_single_calls():
    """The batch and a loop of single-problem FP64 calls give the same ranks
    and values within the FP64 bar."""
    probs = _problems(8, 14, k=4, m_range=(64, 512), n_lo=32, n_hi=300)
    cp = _cp()
    Gs = [to_dev(p.G) for p in probs]
    Fs = [to_dev(p.F) for p in probs]
    Ws, ranks, st = cp.lstsq_batched(Gs, Fs)
    for i, (G, F) in enumerate(zip(Gs, Fs)):
        W1, r1 = cp.lstsq(G, F, mode="fp64")
        assert r1 == ranks[i]
        assert rel(Ws[i].cpu().numpy(), W1.cpu().numpy()) <= TOL["fp64"]


def test_batched_edge_cases():
    """n = 1, m = n, k = 1, G = 0 (r = 0, W = 0), rank 1, a zero column, a
    strided G, and a non-finite problem that fails alone."""
    rng = np.random.default_rng(15)
    cases = []
    cases.append((rng.standard_normal((7, 1)), rng.standard_normal((7, 1))))          # n = 1
    cases.append((rng.standard_normal((33, 33)), rng.standard_normal((33, 2))))       # square
    cases.append((np.zeros((20, 9)), rng.standard_normal((20, 3))))                   # G = 0
    u = rng.standard_normal((50, 1))
    v = rng.standard_normal((1, 17))
    cases.append((u @ v, rng.standard_normal((50, 2))))                                # rank 1
    Gz = rng.standard_normal((40, 12))
    Gz[:, 5] = 0.0
    cases.append((Gz, rng.standard_normal((40, 1))))                                   # zero column
    bad = rng.standard_normal((30, 10))
    bad[3, 4] = np.nan
    cases.append((bad, rng.standard_normal((30, 2))))                                  # non-finite
    cases.append((rng.standard_normal((129, 129)), rng.standard_normal((129, 4))))    # n = 129
    cp = _cp()
    Gs = [to_dev(G) for G, _ in cases]
    # a strided view (ld > n) for one problem
    big = to_dev(np.zeros((40, 20)))
    big[:, :12] = Gs[4]
    Gs[4] = big[:, :12]
    Fs = [to_dev(F) for _, F in cases]
    Ws, ranks, st = cp.lstsq_batched(Gs, Fs)
    for i, (G, F) in enumerate(cases):
        if i == 5:
            assert st[i] == 2 and ranks[i] == -1
            continue
        assert st[i] == 0, (i, st[i])
        r_o, _ = O.rank(G)
        assert ranks[i] == r_o, (i, ranks[i], r_o)
        W_o = O.lstsq(G, F)
        W = Ws[i].cpu().numpy()
        if r_o == 0:
            assert np.all(W == 0.0)
        else:
            assert rel(W, W_o) <= fp64_bar(G, F, r_o), (i, rel(W, W_o))


def test_batched_rejects_unsupported():
    cp = _cp()
    with pytest.raises(cp.CpinvError):
        cp.lstsq_batched([to_dev(np.ones((4, 8)))], [to_dev(np.ones((4, 1)))])  # n > m
    with pytest.raises(cp.CpinvError):
        cp.lstsq_batched([to_dev(np.ones((600, 513)))], [to_dev(np.ones((600, 1)))])  # n > 512


def test_batched_full_workload_sampled():
    """512 problems of the uneven batch workload (m in [64, 1024], n in
    [32, min(m, 512)], r in [n/2, n], k = 4), replayed as a graph: every rank
    equals the construction rank, every W satisfies the normal equations of
    its problem, and 12 sampled problems match the oracle."""
    probs = inputs.batched_problems(512, 4, k=4, attempts=gap.load())
    cp = _cp()
    plan = cp.BatchedLstsq([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs])
    plan()
    Ws, ranks, st = plan()
    Ws, ranks, st = plan()
    assert all(s == 0 for s in st)
    assert ranks == [p.r for p in probs]
    # G'(G W - F) = 0 (the least-squares residual is orthogonal to range(G))
    for i in range(0, 512, 7):
        p = probs[i]
        W = Ws[i].cpu().numpy()
        res = p.G.T @ (p.G @ W - p.F)
        scale = np.linalg.norm(p.G) ** 2 * np.linalg.norm(W) + np.linalg.norm(p.G) * np.linalg.norm(p.F)
        assert np.linalg.norm(res) <= 1e-9 * scale, i
    sample = np.random.default_rng(0).choice(512, size=12, replace=False)
    _check_against_oracle(probs, Ws, ranks, st, idx=sorted(int(i) for i in sample))


# --------------------------------------------------------------------------
# the exact-slice batched mode: every Gram matrix and every L'L of a group
# as one block-diagonal tensor-core residue product (exactly summed, rounded
# once); the factorisation updates, the inverse and the chain stay FP64, so
# the FP64 bar applies
# --------------------------------------------------------------------------

def test_batched_exact_small_uneven():
    probs = _problems(24, 11, k=3, m_range=(16, 300), n_lo=4, n_hi=160)
    cp = _cp()
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     mode="exact")
    _check_against_oracle(probs, Ws, ranks, st)
    assert ranks == [p.r for p in probs]


@pytest.mark.parametrize("panel", [16, 32])
def test_batched_exact_wide_buckets(panel):
    """Groups of n_pad 256 and 512 (where the residue products may take
    256-wide tiles) and ragged m up to the 4096 limit of one exact product."""
    probs = _problems(9, 13, k=2, m_range=(300, 4096), n_lo=130, n_hi=512)
    cp = _cp()
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     mode="exact", panel=panel)
    _check_against_oracle(probs, Ws, ranks, st)


def test_batched_exact_graph_replay_and_fp64_agree():
    probs = _problems(16, 14, k=4, m_range=(64, 700), n_lo=32, n_hi=400)
    cp = _cp()
    Gs, Fs = [to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs]
    plan = cp.BatchedLstsq(Gs, Fs, mode="exact")
    W1 = [w.clone() for w in plan()[0]]
    plan()
    Ws, ranks, st = plan()
    for a, b in zip(W1, Ws):
        assert torch.equal(a, b)
    Wf, rf, _ = cp.lstsq_batched(Gs, Fs, mode="fp64")
    assert rf == ranks
    for p, a, b, r in zip(probs, Ws, Wf, ranks):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 2.0 * fp64_bar(p.G, p.F, r)


def test_batched_exact_rejects_long_problems():
    """m > 4096 exceeds one exact residue product: no workspace size and
    CPINV_ERR_UNSUPPORTED from the call, before any GPU work."""
    import ctypes
    cp = _cp()
    G, F = to_dev(np.ones((4097, 8))), to_dev(np.ones((4097, 1)))
    W = torch.empty((8, 1), dtype=torch.float64, device="cuda:0")
    probs = (cp.Problem * 1)(cp.Problem(4097, 8, 1, G.data_ptr(), 8, F.data_ptr(), 1,
                                        W.data_ptr(), 1))
    o = cp.make_opts("exact")
    assert cp.lib().cpinv_lstsq_batched_workspace_size(1, probs, ctypes.byref(o)) == 0
    ranks = (ctypes.c_int64 * 1)(7)
    status = (ctypes.c_int32 * 1)(0)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda:0")
    rc = cp.lib().cpinv_lstsq_batched(1, probs, ranks, status, ws.data_ptr(), ws.numel(),
                                      ctypes.byref(o), torch.cuda.current_stream().cuda_stream)
    assert rc == 6 and ranks[0] == -1


def test_batched_exact_full_workload():
    """The 512-problem uneven workload in the exact-slice mode: every rank
    equals the construction rank, every W satisfies its normal equations,
    and 32 sampled problems match the oracle."""
    probs = inputs.batched_problems(512, 4, k=4, attempts=gap.load())
    cp = _cp()
    plan = cp.BatchedLstsq([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                           mode="exact")
    plan()
    Ws, ranks, st = plan()
    assert all(s == 0 for s in st)
    assert ranks == [p.r for p in probs]
    for i in range(0, 512, 5):
        p = probs[i]
        W = Ws[i].cpu().numpy()
        res = p.G.T @ (p.G @ W - p.F)
        scale = np.linalg.norm(p.G) ** 2 * np.linalg.norm(W) + np.linalg.norm(p.G) * np.linalg.norm(p.F)
        assert np.linalg.norm(res) <= 1e-9 * scale, i
    sample = np.random.default_rng(1).choice(512, size=32, replace=False)
    _check_against_oracle(probs, Ws, ranks, st, idx=sorted(int(i) for i in sample))


# --------------------------------------------------------------------------
# the factorisations as one persistent launch fed by a device task queue
# (CPINV_BATCH_FACTOR=queue), against the oracle and against the per-panel
# launches
# --------------------------------------------------------------------------

@pytest.fixture
def factor_form(monkeypatch):
    def use(form):
        monkeypatch.setenv("CPINV_BATCH_FACTOR", form)
    return use


@pytest.mark.parametrize("mode", ["fp64", "exact"])
def test_batched_queue_small_uneven(factor_form, mode):
    probs = _problems(24, 11, k=3, m_range=(16, 300), n_lo=4, n_hi=160)
    cp = _cp()
    factor_form("queue")
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     mode=mode)
    _check_against_oracle(probs, Ws, ranks, st)
    assert ranks == [p.r for p in probs]


def test_batched_queue_matches_panel_launches(factor_form):
    """Same batch, both forms of the factorisation: same ranks, and W within
    rounding (the queue applies the same updates in the same panel order,
    tile by tile)."""
    probs = _problems(40, 15, k=4, m_range=(64, 1024), n_lo=32, n_hi=512)
    cp = _cp()
    Gs, Fs = [to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs]
    factor_form("queue")
    Wq, rq, sq = cp.lstsq_batched(Gs, Fs, mode="fp64")
    factor_form("panels")
    Wp, rp, sp = cp.lstsq_batched(Gs, Fs, mode="fp64", panel=32)
    assert all(x == 0 for x in sq + sp)
    assert rq == rp == [p.r for p in probs]
    for p, a, b, r in zip(probs, Wq, Wp, rq):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 2.0 * fp64_bar(p.G, p.F, r)
    sample = list(range(0, 40, 5))
    _check_against_oracle(probs, Wq, rq, sq, idx=sample)


def test_batched_queue_full_workload(factor_form):
    probs = inputs.batched_problems(512, 4, k=4, attempts=gap.load())
    cp = _cp()
    factor_form("queue")
    plan = cp.BatchedLstsq([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                           mode="exact")
    plan()
    Ws, ranks, st = plan()
    assert all(s == 0 for s in st)
    assert ranks == [p.r for p in probs]
    sample = np.random.default_rng(2).choice(512, size=16, replace=False)
    _check_against_oracle(probs, Ws, ranks, st, idx=sorted(int(i) for i in sample))


# --------------------------------------------------------------------------
# the exact mode's left-looking factorisation (CPINV_BATCH_FACTOR=exact):
# every panel's update one block-diagonal residue product over the problems,
# each entry the exact sum rounded once, as in the single-problem path
# --------------------------------------------------------------------------

def test_batched_exact_factor_small_uneven(factor_form):
    probs = _problems(24, 11, k=3, m_range=(16, 300), n_lo=4, n_hi=160)
    cp = _cp()
    factor_form("exact")
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     mode="exact")
    _check_against_oracle(probs, Ws, ranks, st)
    assert ranks == [p.r for p in probs]


def test_batched_exact_factor_wide_buckets(factor_form):
    """n_pad 256 and 512 groups, ragged n and m up to 4096."""
    probs = _problems(9, 13, k=2, m_range=(300, 4096), n_lo=130, n_hi=512)
    cp = _cp()
    factor_form("exact")
    Ws, ranks, st = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                                     mode="exact")
    _check_against_oracle(probs, Ws, ranks, st)


def test_batched_exact_factor_full_workload(factor_form):
    probs = inputs.batched_problems(512, 4, k=4, attempts=gap.load())
    cp = _cp()
    factor_form("exact")
    plan = cp.BatchedLstsq([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs],
                           mode="exact")
    plan()
    Ws, ranks, st = plan()
    assert all(s == 0 for s in st)
    assert ranks == [p.r for p in probs]
    sample = np.random.default_rng(3).choice(512, size=24, replace=False)
    _check_against_oracle(probs, Ws, ranks, st, idx=sorted(int(i) for i in sample))
