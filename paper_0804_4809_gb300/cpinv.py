"""Thin PyTorch binding of libcpinv.so (argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; this module
only checks tensors, allocates outputs and the workspace through PyTorch's
caching allocator, and passes raw device pointers and the current CUDA stream
through the C ABI (``include/cpinv.h``).  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpinv.so")

MODE_FP64 = 0
MODE_EXACT_SLICE = 1
MODE_SPLIT_BF16X3 = 2
_MODES = {"fp64": MODE_FP64, "exact": MODE_EXACT_SLICE, "exact_slice": MODE_EXACT_SLICE,
          "bf16x3": MODE_SPLIT_BF16X3, "split": MODE_SPLIT_BF16X3}

_c_i64 = ctypes.c_int64
_c_vp = ctypes.c_void_p
_c_sz = ctypes.c_size_t


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("panel", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rel_tol", ctypes.c_double)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double)]


class Problem(ctypes.Structure):
    """One problem of a batched least-squares call (``cpinv_problem``)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("G", ctypes.c_void_p), ("ldg", ctypes.c_int64),
                ("F", ctypes.c_void_p), ("ldf", ctypes.c_int64),
                ("W", ctypes.c_void_p), ("ldw", ctypes.c_int64)]


class TimelineEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double)]


class CpinvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cpinv status {status}: {msg}")
        self.status = status


_lib = None

#: Every C symbol ``include/cpinv.h`` declares, with (restype, argtypes).
SIGNATURES = {
    "cpinv_default_opts": (None, [ctypes.POINTER(Opts)]),
    "cpinv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cpinv_version": (ctypes.c_int, []),
    "cpinv_pinv_workspace_size": (_c_sz, [_c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_pinv": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_vp, _c_sz,
                                  ctypes.POINTER(Opts), ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_lstsq_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_lstsq": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64, _c_vp,
                                   _c_i64, _c_vp, _c_sz, ctypes.POINTER(Opts),
                                   ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_rank_workspace_size": (_c_sz, [_c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_rank": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_vp, _c_sz,
                                  ctypes.POINTER(Opts), ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_lstsq_backward_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_lstsq_backward": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64,
                                            _c_vp, _c_i64, _c_vp, _c_i64, _c_vp, _c_i64, _c_vp,
                                            _c_i64, _c_vp, _c_sz, ctypes.POINTER(Opts),
                                            ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_lstsq_state_size": (_c_sz, [_c_i64, _c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_lstsq_forward": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64,
                                           _c_vp, _c_i64, _c_vp, _c_sz, ctypes.POINTER(Opts),
                                           ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_lstsq_backward_from_state": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp,
                                                       _c_i64, _c_i64, _c_vp, _c_i64, _c_vp,
                                                       _c_i64, _c_vp, _c_i64, _c_vp, _c_sz,
                                                       ctypes.POINTER(Opts),
                                                       ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_selftest_wait_timeout": (ctypes.c_int, [_c_vp, _c_sz, _c_vp]),
    "cpinv_selftest_queue_timeout": (ctypes.c_int, [_c_vp, _c_sz, _c_vp]),
    "cpinv_gram_update_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i64, ctypes.c_int32]),
    "cpinv_gram_update": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64,
                                         _c_vp, _c_i64, _c_vp, _c_i64, ctypes.c_int32, _c_vp,
                                         _c_sz, _c_vp]),
    "cpinv_lstsq_gram_workspace_size": (_c_sz, [_c_i64, _c_i64, ctypes.POINTER(Opts)]),
    "cpinv_lstsq_gram": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64, _c_vp,
                                        _c_i64, _c_vp, _c_sz, ctypes.POINTER(Opts),
                                        ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_lstsq_batched_workspace_size": (_c_sz, [ctypes.c_int32, ctypes.POINTER(Problem),
                                                   ctypes.POINTER(Opts)]),
    "cpinv_lstsq_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Problem),
                                           ctypes.POINTER(_c_i64), ctypes.POINTER(ctypes.c_int32),
                                           _c_vp, _c_sz, ctypes.POINTER(Opts), _c_vp]),
    "cpinv_pinv_static": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64,
                                         ctypes.POINTER(Opts), ctypes.POINTER(_c_i64), _c_vp]),
    "cpinv_matmul_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32]),
    "cpinv_matmul": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _c_i64, _c_i64, _c_i64,
                                    ctypes.c_double, _c_vp, _c_i64, _c_vp, _c_i64, ctypes.c_double,
                                    _c_vp, _c_i64, ctypes.c_int32, ctypes.c_int32, _c_vp, _c_sz,
                                    ctypes.c_int32, _c_vp]),
    "cpinv_rbf_design": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64, _c_i64,
                                        ctypes.c_double, _c_vp, _c_i64, _c_vp]),
    "cpinv_rbf_normal_equations_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i64, _c_i64]),
    "cpinv_rbf_normal_equations": (ctypes.c_int, [_c_vp, _c_i64, _c_i64, _c_i64, _c_vp, _c_i64,
                                                  _c_i64, ctypes.c_double, _c_vp, _c_i64, _c_i64,
                                                  _c_vp, _c_i64, _c_vp, _c_i64, _c_vp, _c_sz,
                                                  ctypes.c_int32, _c_vp]),
    "cpinv_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "cpinv_profile_read": (ctypes.c_int, [ctypes.POINTER(ProfileEntry), ctypes.c_int]),
    "cpinv_profile_timeline": (ctypes.c_int, [ctypes.POINTER(TimelineEntry), ctypes.c_int]),
    "cpinv_launch_count": (ctypes.c_int64, []),
}


def lib():
    """Load libcpinv.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def make_opts(mode="fp64", rel_tol: float = 1e-9, panel: int = 0, slices: int = 0) -> Opts:
    o = Opts()
    lib().cpinv_default_opts(ctypes.byref(o))
    o.mode = _MODES[mode] if isinstance(mode, str) else int(mode)
    o.rel_tol = float(rel_tol)
    o.panel = int(panel)
    o.slices = int(slices)
    return o


def _check(status: int):
    if status != 0:
        raise CpinvError(status, lib().cpinv_status_string(status).decode())


def _mat(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or x.dim() != 2:
        raise TypeError(f"{name} must be a 2-D torch tensor")
    if x.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (no CPU path)")
    if x.shape[1] > 1 and x.stride(1) != 1 or x.shape[0] > 1 and x.stride(0) < x.shape[1]:
        x = x.contiguous()
    return x


def _ld(x: torch.Tensor) -> int:
    return max(int(x.stride(0)), int(x.shape[1]), 1) if x.shape[0] > 1 else max(int(x.shape[1]), 1)


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def pinv(G: torch.Tensor, mode="fp64", rel_tol: float = 1e-9, panel: int = 0, slices: int = 0,
         out: torch.Tensor | None = None, sync_rank: bool = True):
    """G+ of a CUDA float64 matrix.  Returns (G+, rank); rank is None when
    ``sync_rank`` is False (no host synchronisation)."""
    G = _mat(G, "G")
    m, n = G.shape
    o = make_opts(mode, rel_tol, panel, slices)
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=G.device)
    ws_bytes = lib().cpinv_pinv_workspace_size(m, n, ctypes.byref(o))
    if ws_bytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    ws = _workspace(ws_bytes, G.device)
    r = _c_i64(-1)
    st = lib().cpinv_pinv(G.data_ptr(), m, n, _ld(G), out.data_ptr(), _ld(out), ws.data_ptr(),
                          ws.numel(), ctypes.byref(o), ctypes.byref(r) if sync_rank else None,
                          _stream(G.device))
    _check(st)
    return out, (int(r.value) if sync_rank else None)


def lstsq(G: torch.Tensor, F: torch.Tensor, mode="fp64", rel_tol: float = 1e-9, panel: int = 0,
          slices: int = 0, out: torch.Tensor | None = None, sync_rank: bool = True):
    """Minimum-norm least squares W = G+ F.  Returns (W, rank)."""
    G = _mat(G, "G")
    F = _mat(F, "F")
    m, n = G.shape
    if F.shape[0] != m:
        raise ValueError("F must have as many rows as G")
    k = F.shape[1]
    o = make_opts(mode, rel_tol, panel, slices)
    if out is None:
        out = torch.empty((n, k), dtype=torch.float64, device=G.device)
    ws_bytes = lib().cpinv_lstsq_workspace_size(m, n, k, ctypes.byref(o))
    if ws_bytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    ws = _workspace(ws_bytes, G.device)
    r = _c_i64(-1)
    st = lib().cpinv_lstsq(G.data_ptr(), m, n, _ld(G), F.data_ptr(), k, _ld(F), out.data_ptr(),
                           _ld(out), ws.data_ptr(), ws.numel(), ctypes.byref(o),
                           ctypes.byref(r) if sync_rank else None, _stream(G.device))
    _check(st)
    return out, (int(r.value) if sync_rank else None)


def rank(G: torch.Tensor, mode="fp64", rel_tol: float = 1e-9, panel: int = 0, slices: int = 0):
    """Numerical rank and kept-pivot mask (uint8, min(m, n) entries)."""
    G = _mat(G, "G")
    m, n = G.shape
    o = make_opts(mode, rel_tol, panel, slices)
    mask = torch.empty((min(m, n),), dtype=torch.uint8, device=G.device)
    ws_bytes = lib().cpinv_rank_workspace_size(m, n, ctypes.byref(o))
    if ws_bytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    ws = _workspace(ws_bytes, G.device)
    r = _c_i64(-1)
    st = lib().cpinv_rank(G.data_ptr(), m, n, _ld(G), mask.data_ptr() if mask.numel() else None,
                          ws.data_ptr(), ws.numel(), ctypes.byref(o), ctypes.byref(r),
                          _stream(G.device))
    _check(st)
    return int(r.value), mask


def gram_update(A: torch.Tensor, G: torch.Tensor, B: torch.Tensor | None = None,
                F: torch.Tensor | None = None, mode="fp64") -> None:
    """A += G'G (lower triangle) and, with F, B += G'F, in place."""
    G = _mat(G, "G")
    m, n = G.shape
    if A.shape != (n, n) or not A.is_contiguous() or A.dtype != torch.float64:
        raise ValueError("A must be a contiguous float64 n x n tensor")
    k = 0
    if F is not None:
        F = _mat(F, "F")
        k = F.shape[1]
        if B is None or B.shape != (n, k) or not B.is_contiguous():
            raise ValueError("B must be a contiguous n x k tensor")
    md = _MODES[mode] if isinstance(mode, str) else int(mode)
    nbytes = lib().cpinv_gram_update_workspace_size(m, n, max(k, 1), md)
    if nbytes == 0:
        raise CpinvError(1, "invalid sizes or mode")
    ws = _workspace(nbytes, G.device)
    st = lib().cpinv_gram_update(G.data_ptr(), m, n, _ld(G),
                                 F.data_ptr() if F is not None else None, k,
                                 _ld(F) if F is not None else 1, A.data_ptr(), n,
                                 B.data_ptr() if B is not None else None, max(k, 1), md,
                                 ws.data_ptr(), ws.numel(), _stream(G.device))
    _check(st)


def lstsq_gram(A: torch.Tensor, B: torch.Tensor, mode="fp64", rel_tol: float = 1e-9,
               panel: int = 0):
    """W = G+ F from normal equations A = G'G (lower triangle read), B = G'F.
    Returns (W, rank)."""
    A = _mat(A, "A")
    B = _mat(B, "B")
    n, k = A.shape[0], B.shape[1]
    o = make_opts(mode, rel_tol, panel)
    if A.shape != (n, n) or B.shape[0] != n:
        raise ValueError("A must be n x n and B n x k")
    W = torch.zeros((n, k), dtype=torch.float64, device=A.device)
    if n == 0:
        return W, 0
    nbytes = lib().cpinv_lstsq_gram_workspace_size(n, k, ctypes.byref(o))
    if nbytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    ws = _workspace(nbytes, A.device)
    r = _c_i64(-1)
    st = lib().cpinv_lstsq_gram(A.data_ptr(), n, _ld(A), B.data_ptr(), k, _ld(B), W.data_ptr(),
                                _ld(W), ws.data_ptr(), ws.numel(), ctypes.byref(o),
                                ctypes.byref(r), _stream(A.device))
    _check(st)
    return W, int(r.value)


def rbf_design(X: torch.Tensor, C: torch.Tensor, width: float,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Gaussian RBF design matrix G_ij = exp(-|x_i - c_j|^2 / (2 width^2)),
    m x n, computed on the GPU (``cpinv_rbf_design``)."""
    X = _mat(X, "X")
    C = _mat(C, "C")
    m, d = X.shape
    n = C.shape[0]
    if C.shape[1] != d:
        raise ValueError("X and C must have the same number of columns")
    G = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=X.device)
    if G.shape != (m, n) or not G.is_contiguous() or G.dtype != torch.float64:
        raise ValueError("out must be a contiguous float64 m x n tensor")
    st = lib().cpinv_rbf_design(X.data_ptr(), m, d, _ld(X), C.data_ptr(), n, _ld(C),
                                float(width), G.data_ptr(), n, _stream(X.device))
    _check(st)
    return G


def rbf_normal_equations(X: torch.Tensor, C: torch.Tensor, width: float,
                         F: torch.Tensor | None = None, A: torch.Tensor | None = None,
                         B: torch.Tensor | None = None, check: bool = True):
    """A = G'G (lower triangle) and, with F, B = G'F for the RBF design
    matrix G of (X, C, width), without G in memory (exact-slice arithmetic,
    ``cpinv_rbf_normal_equations``).  Returns (A, B)."""
    X = _mat(X, "X")
    C = _mat(C, "C")
    m, d = X.shape
    n = C.shape[0]
    k = 0
    if F is not None:
        F = _mat(F, "F")
        k = F.shape[1]
        if F.shape[0] != m:
            raise ValueError("F must have m rows")
    if A is None:
        A = torch.zeros((n, n), dtype=torch.float64, device=X.device)
    if F is not None and B is None:
        B = torch.zeros((n, k), dtype=torch.float64, device=X.device)
    nbytes = lib().cpinv_rbf_normal_equations_workspace_size(m, n, d, k)
    if nbytes == 0:
        raise CpinvError(6, "unsupported sizes")
    ws = _workspace(nbytes, X.device)
    st = lib().cpinv_rbf_normal_equations(
        X.data_ptr(), m, d, _ld(X), C.data_ptr(), n, _ld(C), float(width),
        F.data_ptr() if F is not None else None, k, _ld(F) if F is not None else 1,
        A.data_ptr(), _ld(A), B.data_ptr() if B is not None else None,
        _ld(B) if B is not None else 1, ws.data_ptr(), ws.numel(), 1 if check else 0,
        _stream(X.device))
    _check(st)
    return A, B


def selftest_wait_timeout(device=None) -> int:
    """Runs the kernels' bounded wait on a counter nothing advances; returns
    the library status (CPINV_ERR_TIMEOUT expected)."""
    import torch
    dev = torch.device("cuda", 0) if device is None else torch.device(device)
    ws = _workspace(256, dev)
    return int(lib().cpinv_selftest_wait_timeout(ws.data_ptr(), ws.numel(), _stream(dev)))


def selftest_queue_timeout(device=None) -> int:
    """Runs the batched queue's bounded wait on an input no task produces;
    returns the library status (CPINV_ERR_TIMEOUT expected)."""
    dev = torch.device("cuda", 0) if device is None else torch.device(device)
    ws = _workspace(64 * 1024, dev)
    return int(lib().cpinv_selftest_queue_timeout(ws.data_ptr(), ws.numel(), _stream(dev)))


def lstsq_backward(G: torch.Tensor, F: torch.Tensor, dW: torch.Tensor, mode="fp64",
                   rel_tol: float = 1e-9, panel: int = 0, slices: int = 0, need_dF: bool = True,
                   need_W: bool = False):
    """Adjoint of W = G+ F: returns (dG, dF or None, W or None, rank) for the
    cotangent dW = dL/dW, the kept-pivot set held fixed (m >= n)."""
    G = _mat(G, "G")
    F = _mat(F, "F")
    dW = _mat(dW, "dW")
    m, n = G.shape
    k = F.shape[1]
    if F.shape[0] != m or tuple(dW.shape) != (n, k):
        raise ValueError("shapes: G m x n, F m x k, dW n x k")
    o = make_opts(mode, rel_tol, panel, slices)
    dG = torch.empty((m, n), dtype=torch.float64, device=G.device)
    dF = torch.empty((m, k), dtype=torch.float64, device=G.device) if need_dF else None
    W = torch.empty((n, k), dtype=torch.float64, device=G.device) if need_W else None
    ws_bytes = lib().cpinv_lstsq_backward_workspace_size(m, n, k, ctypes.byref(o))
    if ws_bytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    ws = _workspace(ws_bytes, G.device)
    r = _c_i64(-1)
    st = lib().cpinv_lstsq_backward(
        G.data_ptr(), m, n, _ld(G), F.data_ptr(), k, _ld(F), dW.data_ptr(), _ld(dW),
        dG.data_ptr(), _ld(dG), dF.data_ptr() if dF is not None else None,
        _ld(dF) if dF is not None else max(k, 1), W.data_ptr() if W is not None else None,
        _ld(W) if W is not None else max(k, 1), ws.data_ptr(), ws.numel(), ctypes.byref(o),
        ctypes.byref(r), _stream(G.device))
    _check(st)
    return dG, dF, W, int(r.value)


def lstsq_forward(G: torch.Tensor, F: torch.Tensor, mode="fp64", rel_tol: float = 1e-9,
                  panel: int = 0):
    """W = G+ F (m >= n) keeping the forward factors for a later reverse
    pass (``cpinv_lstsq_forward``).  Returns (W, rank, state); the state is
    a device buffer for ``lstsq_backward_from_state``."""
    G = _mat(G, "G")
    F = _mat(F, "F")
    m, n = G.shape
    k = F.shape[1]
    if F.shape[0] != m:
        raise ValueError("F must have m rows")
    o = make_opts(mode, rel_tol, panel)
    nbytes = lib().cpinv_lstsq_state_size(m, n, k, ctypes.byref(o))
    if nbytes == 0:
        raise CpinvError(1, "invalid options or sizes")
    state = _workspace(nbytes, G.device)
    W = torch.empty((n, k), dtype=torch.float64, device=G.device)
    r = _c_i64(-1)
    st = lib().cpinv_lstsq_forward(G.data_ptr(), m, n, _ld(G), F.data_ptr(), k, _ld(F),
                                   W.data_ptr(), _ld(W), state.data_ptr(), state.numel(),
                                   ctypes.byref(o), ctypes.byref(r), _stream(G.device))
    _check(st)
    return W, int(r.value), state


def lstsq_backward_from_state(G: torch.Tensor, F: torch.Tensor, dW: torch.Tensor,
                              state: torch.Tensor, mode="fp64", rel_tol: float = 1e-9,
                              panel: int = 0, need_dF: bool = True):
    """The adjoint of W = G+ F from the factors ``lstsq_forward`` kept
    (``cpinv_lstsq_backward_from_state``): returns (dG, dF or None, rank)."""
    G = _mat(G, "G")
    F = _mat(F, "F")
    dW = _mat(dW, "dW")
    m, n = G.shape
    k = F.shape[1]
    if F.shape[0] != m or tuple(dW.shape) != (n, k):
        raise ValueError("shapes: G m x n, F m x k, dW n x k")
    o = make_opts(mode, rel_tol, panel)
    dG = torch.empty((m, n), dtype=torch.float64, device=G.device)
    dF = torch.empty((m, k), dtype=torch.float64, device=G.device) if need_dF else None
    r = _c_i64(-1)
    st = lib().cpinv_lstsq_backward_from_state(
        G.data_ptr(), m, n, _ld(G), F.data_ptr(), k, _ld(F), dW.data_ptr(), _ld(dW),
        dG.data_ptr(), _ld(dG), dF.data_ptr() if dF is not None else None,
        _ld(dF) if dF is not None else max(k, 1), state.data_ptr(), state.numel(),
        ctypes.byref(o), ctypes.byref(r), _stream(G.device))
    _check(st)
    return dG, dF, int(r.value)


class LstsqFunction(torch.autograd.Function):
    """W = G+ F as a differentiable op: forward through cpinv_lstsq_forward,
    which keeps the factors L, (L'L)^-1, the kept-pivot set and the rank, and
    backward through the hand-written adjoint from those factors
    (cpinv_lstsq_backward_from_state; kept-pivot set held fixed), so a
    training step factors once.  Wide G (m < n) goes through cpinv_lstsq and
    the recomputing adjoint's error (unsupported)."""

    @staticmethod
    def forward(ctx, G, F, mode="fp64", rel_tol=1e-9):
        ctx.mode = mode
        ctx.rel_tol = rel_tol
        if G.shape[0] >= G.shape[1] > 0 and F.shape[1] > 0:
            W, r, state = lstsq_forward(G, F, mode=mode, rel_tol=rel_tol)
            ctx.state = state
        else:
            W, r = lstsq(G, F, mode=mode, rel_tol=rel_tol)
            ctx.state = None
        ctx.save_for_backward(G, F)
        ctx.rank = r
        return W

    @staticmethod
    def backward(ctx, dW):
        G, F = ctx.saved_tensors
        need_G, need_F = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_G or need_F):
            return None, None, None, None
        if ctx.state is not None:
            dG, dF, _ = lstsq_backward_from_state(G, F, dW.contiguous(), ctx.state,
                                                  mode=ctx.mode, rel_tol=ctx.rel_tol,
                                                  need_dF=need_F)
            ctx.state = None  # one reverse pass per forward
        else:
            dG, dF, _, _ = lstsq_backward(G, F, dW.contiguous(), mode=ctx.mode,
                                          rel_tol=ctx.rel_tol, need_dF=need_F)
        return (dG if need_G else None), dF, None, None


def lstsq_autograd(G: torch.Tensor, F: torch.Tensor, mode="fp64", rel_tol: float = 1e-9):
    """Differentiable W = G+ F (see ``LstsqFunction``)."""
    return LstsqFunction.apply(G, F, mode, rel_tol)


class BatchedLstsq:
    """W_p = G_p+ F_p for a list of problems of uneven size, as one batch.

    The descriptor array, the outputs and the workspace are built once, so
    repeated calls with the same tensors replay one CUDA graph of the whole
    batch.  ``Gs``/``Fs`` are lists of CUDA float64 matrices (m_p x n_p with
    n_p <= m_p, and m_p x k_p).  ``mode``: "fp64", or "exact" (the Gram and
    L'L products of every problem on the tensor cores, exactly summed and
    rounded once; m_p <= 4096)."""

    def __init__(self, Gs, Fs, rel_tol: float = 1e-9, panel: int = 0, mode="fp64"):
        if len(Gs) != len(Fs):
            raise ValueError("Gs and Fs differ in length")
        self.Gs = [_mat(G, "G") for G in Gs]
        self.Fs = [_mat(F, "F") for F in Fs]
        self.P = len(self.Gs)
        self.device = self.Gs[0].device if self.P else torch.device("cuda")
        self.opts = make_opts(mode, rel_tol, panel)
        self.Ws = []
        self.probs = (Problem * max(self.P, 1))()
        for i, (G, F) in enumerate(zip(self.Gs, self.Fs)):
            m, n = G.shape
            if F.shape[0] != m:
                raise ValueError(f"problem {i}: F must have as many rows as G")
            W = torch.empty((n, F.shape[1]), dtype=torch.float64, device=G.device)
            self.Ws.append(W)
            self.probs[i] = Problem(m, n, F.shape[1], G.data_ptr(), _ld(G), F.data_ptr(), _ld(F),
                                    W.data_ptr(), _ld(W))
        nbytes = lib().cpinv_lstsq_batched_workspace_size(self.P, self.probs,
                                                          ctypes.byref(self.opts))
        if nbytes == 0 and self.P:
            raise CpinvError(1, "invalid or unsupported problem sizes")
        self.ws = _workspace(nbytes, self.device)
        self.ranks = (_c_i64 * max(self.P, 1))()
        self.status = (ctypes.c_int32 * max(self.P, 1))()

    def __call__(self, sync: bool = True, stream: int | None = None):
        """Runs the batch; with ``sync`` returns (Ws, ranks, statuses)."""
        st = lib().cpinv_lstsq_batched(self.P, self.probs, self.ranks if sync else None,
                                       self.status if sync else None, self.ws.data_ptr(),
                                       self.ws.numel(), ctypes.byref(self.opts),
                                       _stream(self.device) if stream is None else stream)
        if not sync:
            _check(st)
            return self.Ws, None, None
        statuses = [int(self.status[i]) for i in range(self.P)]
        if st != 0 and all(x == 0 for x in statuses):
            _check(st)
        return self.Ws, [int(self.ranks[i]) for i in range(self.P)], statuses


def lstsq_batched(Gs, Fs, rel_tol: float = 1e-9, panel: int = 0, mode="fp64"):
    """One batched call: returns (Ws, ranks, statuses) (see ``BatchedLstsq``)."""
    return BatchedLstsq(Gs, Fs, rel_tol, panel, mode)()


def profile_enable(on: bool = True) -> bool:
    """Turn the library's per-launch CUDA-event tracing on or off (clears it)."""
    return bool(lib().cpinv_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """Per kernel class: {'launches', 'ms', 'flops'} since the last read."""
    arr = (ProfileEntry * 16)()
    n = lib().cpinv_profile_read(arr, 16)
    if n < 0:
        raise CpinvError(4, "profile read failed")
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].ms),
                                   "flops": float(arr[i].flops)} for i in range(min(n, 16))}


def profile_timeline(max_entries: int = 100000) -> list:
    """Per traced launch (launch order): (class, start_ms, end_ms) relative
    to the first traced launch.  Call before ``profile_read``."""
    arr = (TimelineEntry * max_entries)()
    n = lib().cpinv_profile_timeline(arr, max_entries)
    if n < 0:
        raise CpinvError(4, "profile timeline failed")
    return [(arr[i].name.decode(), float(arr[i].start_ms), float(arr[i].end_ms))
            for i in range(min(n, max_entries))]


def launch_count() -> int:
    """Kernels launched by the library in this process."""
    return int(lib().cpinv_launch_count())


class PinvPlan:
    """Pre-sized G+ call for repeated use: the workspace is allocated once."""

    def __init__(self, m: int, n: int, device, mode="fp64", rel_tol: float = 1e-9,
                 panel: int = 0, slices: int = 0):
        self.m, self.n = int(m), int(n)
        self.device = torch.device(device)
        self.opts = make_opts(mode, rel_tol, panel, slices)
        nbytes = lib().cpinv_pinv_workspace_size(self.m, self.n, ctypes.byref(self.opts))
        if nbytes == 0:
            raise CpinvError(1, "invalid options or sizes")
        self.ws = _workspace(nbytes, self.device)

    def __call__(self, G: torch.Tensor, out: torch.Tensor, sync_rank: bool = False,
                 stream: int | None = None):
        r = _c_i64(-1)
        st = lib().cpinv_pinv(G.data_ptr(), self.m, self.n, _ld(G), out.data_ptr(), _ld(out),
                              self.ws.data_ptr(), self.ws.numel(), ctypes.byref(self.opts),
                              ctypes.byref(r) if sync_rank else None,
                              _stream(self.device) if stream is None else stream)
        _check(st)
        return int(r.value) if sync_rank else None


def matmul(A: torch.Tensor, B: torch.Tensor, transA: bool = False, transB: bool = False,
           mode="fp64", bits: int = 0, alpha: float = 1.0, beta: float = 0.0,
           C: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C in the library's arithmetic (FP64 or
    exact-slice residue products on the tensor cores)."""
    A = _mat(A, "A")
    B = _mat(B, "B")
    M, K = (A.shape[1], A.shape[0]) if transA else (A.shape[0], A.shape[1])
    K2, N = (B.shape[1], B.shape[0]) if transB else (B.shape[0], B.shape[1])
    if K != K2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    md = _MODES[mode] if isinstance(mode, str) else int(mode)
    sym = int(A.data_ptr() == B.data_ptr() and transA != transB and M == N)
    nbytes = lib().cpinv_matmul_workspace_size(M, N, K, md, bits, sym)
    if nbytes == 0:
        raise CpinvError(1, "invalid sizes or options")
    ws = _workspace(nbytes, A.device)
    st = lib().cpinv_matmul(int(transA), int(transB), M, N, K, float(alpha), A.data_ptr(), _ld(A),
                            B.data_ptr(), _ld(B), float(beta), C.data_ptr(), _ld(C), md, int(bits),
                            ws.data_ptr(), ws.numel(), int(check), _stream(A.device))
    _check(st)
    return C
