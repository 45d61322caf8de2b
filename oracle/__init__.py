"""CPU FP64 oracle for the full-rank-Cholesky Moore-Penrose inverse.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may
import anything from this package.  It shares no code with the CUDA library.
"""
from .geninv import (REL_TOL, exact_cross, full_rank_cholesky, geninv, gram, lstsq,
                     lstsq_from_gram, penrose_residuals, pivot_tolerance, rank)
from .adjoint import golub_pereyra_vjp, lstsq_vjp

__all__ = ["REL_TOL", "exact_cross", "gram", "pivot_tolerance", "full_rank_cholesky",
           "geninv", "rank", "lstsq", "penrose_residuals", "lstsq_vjp", "golub_pereyra_vjp", "lstsq_from_gram"]
