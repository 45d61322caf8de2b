"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol ``include/cpinv.h`` declares; host-only argument validation and
workspace sizing behave as documented.  No call here touches a GPU."""
import ctypes
import os
import re

import pytest

from paper_0804_4809_gb300 import build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv.lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "cpinv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(cpinv_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for must in ["cpinv_pinv", "cpinv_lstsq", "cpinv_rank", "cpinv_pinv_workspace_size",
                 "cpinv_lstsq_workspace_size", "cpinv_rank_workspace_size",
                 "cpinv_default_opts", "cpinv_status_string", "cpinv_version"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_0804_4809_gb300 import cpinv
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in cpinv.SIGNATURES, name


def test_default_opts_and_status_strings(lib):
    from paper_0804_4809_gb300 import cpinv
    o = cpinv.Opts()
    lib.cpinv_default_opts(ctypes.byref(o))
    assert o.mode == 0 and o.rel_tol == 1e-9 and o.panel == 0 and o.reserved == 0
    assert lib.cpinv_status_string(0) == b"ok"
    assert b"non-finite" in lib.cpinv_status_string(2)
    assert lib.cpinv_version() >= 100


def test_workspace_sizes(lib):
    from paper_0804_4809_gb300 import cpinv
    o = cpinv.make_opts("fp64")
    s_rank = lib.cpinv_rank_workspace_size(4096, 2048, ctypes.byref(o))
    s_pinv = lib.cpinv_pinv_workspace_size(4096, 2048, ctypes.byref(o))
    s_lsq = lib.cpinv_lstsq_workspace_size(4096, 2048, 16, ctypes.byref(o))
    assert 2048 * 2048 * 8 <= s_rank < s_pinv < s_lsq
    # the transposed branch factors the m x m Gram matrix
    assert lib.cpinv_pinv_workspace_size(2048, 4096, ctypes.byref(o)) == s_pinv
    assert lib.cpinv_pinv_workspace_size(-1, 5, ctypes.byref(o)) == 0
    bad = cpinv.make_opts("fp64", panel=33)
    assert lib.cpinv_pinv_workspace_size(10, 5, ctypes.byref(bad)) == 0


def test_host_side_argument_errors(lib):
    """Argument errors are reported before any CUDA call."""
    from paper_0804_4809_gb300 import cpinv
    o = cpinv.make_opts("fp64")
    r = ctypes.c_int64(7)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    # ld too small
    assert lib.cpinv_pinv(fake, 10, 5, 4, fake, 10, fake, 1 << 20, ctypes.byref(o), ctypes.byref(r), None) == 1
    assert r.value == -1
    # negative size
    assert lib.cpinv_pinv(fake, -1, 5, 5, fake, 10, fake, 1 << 20, ctypes.byref(o), ctypes.byref(r), None) == 1
    # NULL G
    assert lib.cpinv_pinv(None, 10, 5, 5, fake, 10, fake, 1 << 20, ctypes.byref(o), ctypes.byref(r), None) == 1
    # misaligned / missing / small workspace
    assert lib.cpinv_pinv(fake, 10, 5, 5, fake, 10, ctypes.c_void_p(0x1001), 1 << 20, ctypes.byref(o), ctypes.byref(r), None) == 3
    assert lib.cpinv_pinv(fake, 10, 5, 5, fake, 10, None, 1 << 20, ctypes.byref(o), ctypes.byref(r), None) == 3
    assert lib.cpinv_pinv(fake, 10, 5, 5, fake, 10, fake, 16, ctypes.byref(o), ctypes.byref(r), None) == 3
    # bad options
    bad = cpinv.make_opts("fp64", panel=100)
    assert lib.cpinv_pinv(fake, 10, 5, 5, fake, 10, fake, 1 << 20, ctypes.byref(bad), ctypes.byref(r), None) == 1
    bad = cpinv.make_opts("fp64")
    bad.reserved = 3
    assert lib.cpinv_lstsq(fake, 10, 5, 5, fake, 2, 2, fake, 2, fake, 1 << 20, ctypes.byref(bad), ctypes.byref(r), None) == 1
    bad = cpinv.make_opts("fp64", rel_tol=float("nan"))
    assert lib.cpinv_rank(fake, 10, 5, 5, None, fake, 1 << 20, ctypes.byref(bad), ctypes.byref(r), None) == 1
    bad = cpinv.make_opts(9)
    assert lib.cpinv_rank(fake, 10, 5, 5, None, fake, 1 << 20, ctypes.byref(bad), ctypes.byref(r), None) == 1


def test_empty_sizes_need_no_gpu(lib):
    from paper_0804_4809_gb300 import cpinv
    o = cpinv.make_opts("fp64")
    r = ctypes.c_int64(7)
    for m, n in [(0, 0), (0, 5), (5, 0)]:
        assert lib.cpinv_pinv(None, m, n, max(n, 1), None, max(m, 1), None, 0, ctypes.byref(o), ctypes.byref(r), None) == 0
        assert r.value == 0
        assert lib.cpinv_rank(None, m, n, max(n, 1), None, None, 0, ctypes.byref(o), ctypes.byref(r), None) == 0
        assert r.value == 0


def test_batched_argument_checks_need_no_gpu(lib):
    """cpinv_lstsq_batched validates every descriptor and option on the host
    before any CUDA call."""
    from paper_0804_4809_gb300 import cpinv
    o = cpinv.make_opts("fp64")
    fake = ctypes.c_void_p(0x100000)
    P = cpinv.Problem

    def arr(*ps):
        a = (P * len(ps))()
        for i, p in enumerate(ps):
            a[i] = p
        return a

    good = P(100, 40, 4, fake, 40, fake, 4, fake, 4)
    ws = lib.cpinv_lstsq_batched_workspace_size(1, arr(good), ctypes.byref(o))
    assert ws > 100 * 40 * 8
    # two problems in different n buckets need more than one
    ws2 = lib.cpinv_lstsq_batched_workspace_size(2, arr(good, P(600, 300, 4, fake, 300, fake, 4, fake, 4)),
                                                 ctypes.byref(o))
    assert ws2 > ws
    assert lib.cpinv_lstsq_batched(0, None, None, None, None, 0, ctypes.byref(o), None) == 0
    assert lib.cpinv_lstsq_batched(1, None, None, None, fake, 1 << 30, ctypes.byref(o), None) == 1
    ranks = (ctypes.c_int64 * 1)(5)
    status = (ctypes.c_int32 * 1)(0)
    cases = [
        (P(100, 40, 4, None, 40, fake, 4, fake, 4), 1),     # G NULL
        (P(100, 40, 4, fake, 39, fake, 4, fake, 4), 1),     # ldg < n
        (P(100, 40, 0, fake, 40, fake, 4, fake, 4), 1),     # k = 0
        (P(100, 40, 4, fake, 40, fake, 4, fake, 3), 1),     # ldw < k
        (P(30, 40, 4, fake, 40, fake, 4, fake, 4), 6),      # n > m
        (P(900, 513, 4, fake, 513, fake, 4, fake, 4), 6),   # n > 512
        (P(900, 40, 257, fake, 40, fake, 257, fake, 257), 6),  # k > 256
    ]
    for p, code in cases:
        assert lib.cpinv_lstsq_batched(1, arr(p), ranks, status, fake, 1 << 30, ctypes.byref(o), None) == code
        assert ranks[0] == -1
        assert lib.cpinv_lstsq_batched_workspace_size(1, arr(p), ctypes.byref(o)) == 0
    # the split tier is not offered in the batch; the exact-slice mode is,
    # for m <= 4096 (one exact residue product)
    sp = cpinv.make_opts("bf16x3")
    assert lib.cpinv_lstsq_batched(1, arr(good), None, None, fake, 1 << 30, ctypes.byref(sp), None) == 6
    ex = cpinv.make_opts("exact")
    long_ = P(5000, 40, 4, fake, 40, fake, 4, fake, 4)
    assert lib.cpinv_lstsq_batched(1, arr(long_), None, None, fake, 1 << 30, ctypes.byref(ex), None) == 6
    assert lib.cpinv_lstsq_batched_workspace_size(1, arr(long_), ctypes.byref(ex)) == 0
    # the exact-slice batch needs more workspace (residue planes and products)
    assert lib.cpinv_lstsq_batched_workspace_size(1, arr(good), ctypes.byref(ex)) > ws
    bad_panel = cpinv.make_opts("fp64", panel=24)
    assert lib.cpinv_lstsq_batched(1, arr(good), None, None, fake, 1 << 30, ctypes.byref(bad_panel), None) == 1
    # workspace misaligned or too small
    assert lib.cpinv_lstsq_batched(1, arr(good), None, None, ctypes.c_void_p(0x100010), 1 << 30,
                                   ctypes.byref(o), None) == 3
    assert lib.cpinv_lstsq_batched(1, arr(good), None, None, fake, ws - 256, ctypes.byref(o), None) == 3
