"""The allocation-free entry point cpinv_pinv_static, called through the C ABI.

It exists for callers that cannot allocate device memory (a real-time loop in
which cudaMalloc / cudaFree would block or synchronize the device, a plugin
whose host application owns all GPU memory); its scratch is a fixed 1 MiB
device array inside the library.  These checks compare it with the regular
entry point cpinv_pinv on two calls in a row -- the second call reuses the
array the first one left behind -- and with the CPU oracle, and check the
documented limits: orders above 128 and modes whose workspace does not fit
in the array (the exact-slice mode at any size) are refused before any GPU
work.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs

from gpu_util import TOL, rel, tol_for

pytestmark = pytest.mark.gpu

UNSUPPORTED = 6  # CPINV_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_4809_gb300 import build
    build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _static_pinv(cp, G_dev, mode="fp64"):
    import torch
    m, n = G_dev.shape
    out = torch.full((n, m), float("nan"), dtype=torch.float64, device=G_dev.device)
    o = cp.make_opts(mode)
    r = ctypes.c_int64(-1)
    st = cp.lib().cpinv_pinv_static(G_dev.data_ptr(), m, n, n, out.data_ptr(), m, ctypes.byref(o),
                                    ctypes.byref(r), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, int(r.value), out.cpu().numpy()


def test_static_matches_regular_entry_point_twice(cp):
    import torch
    dev = torch.device("cuda:0")
    cases = [inputs.rank_deficient(120, 100, 70, seed=31),   # tall, ragged panels
             inputs.rank_deficient(60, 128, 45, seed=32)]    # wide: transposed branch, order 60
    for G in cases:
        Gd = torch.from_numpy(G).to(dev)
        Yref, rref = cp.pinv(Gd, mode="fp64")
        torch.cuda.synchronize()
        Yo, fac = oracle.geninv(G, return_factors=True)
        for _ in range(2):
            st, r, Y = _static_pinv(cp, Gd)
            assert st == 0, cp.lib().cpinv_status_string(st)
            assert r == rref == fac["rank"]
            assert rel(Y, Yref.cpu().numpy()) <= TOL["fp64"]
            assert rel(Y, Yo) <= tol_for("fp64", G, fac["rank"])


def test_static_rejects_sizes_over_the_limit(cp):
    import torch
    G = torch.zeros((200, 129), dtype=torch.float64, device="cuda:0")
    st, r, _ = _static_pinv(cp, G)
    assert st == UNSUPPORTED and r == -1          # nothing computed
    G = torch.zeros((129, 300), dtype=torch.float64, device="cuda:0")
    st, r, _ = _static_pinv(cp, G)
    assert st == UNSUPPORTED


def test_static_refuses_modes_that_do_not_fit(cp):
    """The exact-slice mode's workspace exceeds the array at every size and
    BF16x3's does above order ~32: refused before any GPU work (the output
    keeps its NaN fill); a BF16x3 call that fits runs and equals the regular
    entry point's result."""
    import torch
    dev = torch.device("cuda:0")
    for shape, mode in (((40, 20), "exact"), ((120, 100), "exact"), ((120, 100), "bf16x3")):
        o = cp.make_opts(mode)
        assert cp.lib().cpinv_pinv_workspace_size(shape[0], shape[1], ctypes.byref(o)) > (1 << 20)
        G = torch.from_numpy(inputs.rank_deficient(shape[0], shape[1], shape[1] // 2, seed=33)).to(dev)
        st, r, Y = _static_pinv(cp, G, mode)
        assert st == UNSUPPORTED and r == -1, (shape, mode, st)
        assert np.all(np.isnan(Y))
    G = inputs.rank_deficient(40, 20, 12, seed=34)
    o = cp.make_opts("bf16x3")
    assert cp.lib().cpinv_pinv_workspace_size(40, 20, ctypes.byref(o)) <= (1 << 20)
    Gd = torch.from_numpy(G).to(dev)
    Yref, rref = cp.pinv(Gd, mode="bf16x3")
    torch.cuda.synchronize()
    st, r, Y = _static_pinv(cp, Gd, "bf16x3")
    assert st == 0 and r == rref
    assert rel(Y, Yref.cpu().numpy()) <= 1e-12
