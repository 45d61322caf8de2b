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
    bad = cpinv.make_opts("fp64", panel=65)
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
