"""GB300-native full-rank-Cholesky Moore-Penrose inverse (Courrieu's method).

The compute path lives in the CUDA shared library ``libcpinv.so`` (sources in
``csrc/``, C ABI in ``include/cpinv.h``).  ``paper_0804_4809_gb300.cpinv`` is
the thin PyTorch binding; submodules are imported lazily so that the seeded
input generators (``inputs``) can be used without a GPU or a built library.
"""
import importlib

__all__ = ["cpinv", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
