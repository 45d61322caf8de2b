"""Failure detection on the GPU without a fault: the factorisation kernels'
bounded wait, run on a counter that nothing advances, must give up, report
CPINV_ERR_TIMEOUT to the host and leave the context usable."""
import time

import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs

from gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu

CPINV_ERR_TIMEOUT = 7  # include/cpinv.h


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_4809_gb300 import build
    build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def test_bounded_wait_expires_and_context_survives(cp):
    import torch
    t0 = time.time()
    st = cp.selftest_wait_timeout()
    elapsed = time.time() - t0
    assert st == CPINV_ERR_TIMEOUT
    assert cp.lib().cpinv_status_string(st).decode() == "a device-side wait timed out"
    assert elapsed < 30.0
    # the context still runs the factorisation
    G = inputs.workload_small()
    Y, r = cp.pinv(to_dev(G), mode="exact")
    torch.cuda.synchronize()
    assert r == 80
    assert rel(Y.cpu().numpy(), oracle.geninv(G)) < 1e-10
    assert np.isfinite(Y.cpu().numpy()).all()


def test_queue_wait_expires_and_context_survives(cp):
    """The batched path's task queue: a task whose input no task produces
    waits (bounded), records the timeout, raises the abort flag and the
    launch ends; the context then still solves a batch."""
    import torch
    t0 = time.time()
    st = cp.selftest_queue_timeout()
    assert st == CPINV_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    probs = inputs.batched_problems(3, seed=7, k=2, m_range=(40, 90), n_lo=10, n_hi=40)
    Ws, ranks, sts = cp.lstsq_batched([to_dev(p.G) for p in probs], [to_dev(p.F) for p in probs])
    torch.cuda.synchronize()
    for p, W, r, s in zip(probs, Ws, ranks, sts):
        assert s == 0 and r == oracle.rank(p.G)[0]
        assert rel(W.cpu().numpy(), oracle.lstsq(p.G, p.F)) < 1e-9
