"""Batched band (tridiagonal / pentadiagonal) solvers on NVIDIA GB300.

The methods of Veneva & Ayriyan, "Performance Analysis of Effective Methods for
Solving Band Matrix SLAEs after Parabolic Nonlinear PDEs" (arXiv:1804.09666) --
NTDM/NPDM, STDM/SPDM, SIP with ILU(0) and Hotelling-Bodewig -- plus FP32 +
refinement and an adjoint, as hand-written sm_103a CUDA kernels behind the C ABI
of include/band.h.  This package is the thin Python binding over torch CUDA tensors.
"""
from ._lib import BandError, load  # noqa: F401
from .band import (AdiStepper, BandSolve, BatchPlan, RaggedPlan, adjoint, desc_for, det, factor,  # noqa: F401
                   refine_solve, sip, sip2d, slogdet, solve, solve_batch, solve_ragged, status_names)

__all__ = ["AdiStepper", "solve", "solve_ragged", "solve_batch", "BatchPlan", "RaggedPlan", "factor", "sip",
           "refine_solve", "sip2d", "adjoint", "det", "slogdet", "BandSolve", "desc_for", "status_names", "load",
           "BandError"]
