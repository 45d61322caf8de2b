"""The allocation-free entry point cpinv_pinv_static, called through the C ABI.

It exists for callers that cannot allocate device memory (a real-time loop in
which cudaMalloc / cudaFree would block or synchronize the device, a plugin
whose host application owns all GPU memory); its scratch is a fixed 1 MiB
device array inside the library.  These checks compare it with the regular
entry point cpinv_pinv on two calls in a row -- the second call reuses the
array the first one left behind -- and check the documented size limit.  The
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_0804_4809_gb300 import inputs

from gpu_util import TOL, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_4809_gb300 import build
    build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _static_pinv(cp, G_dev):
    import torch
    m, n = G_dev.shape
    out = torch.full((n, m), float("nan"), dtype=torch.float64, device=G_dev.device)
    o = cp.make_opts("fp64")
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
        st, r, Y = _static_pinv(cp, Gd)
        assert st == 0, cp.lib().cpinv_status_string(st)
        assert r == rref
        assert rel(Y, Yref.cpu().numpy()) <= TOL["fp64"]


def test_static_rejects_sizes_over_the_limit(cp):
    import torch
    G = torch.zeros((200, 129), dtype=torch.float64, device="cuda:0")
    st, r, _ = _static_pinv(cp, G)
    assert st == 6 and r == -1          # CPINV_ERR_UNSUPPORTED, nothing computed
    G = torch.zeros((129, 300), dtype=torch.float64, device="cuda:0")
    st, r, _ = _static_pinv(cp, G)
    assert st == 6
