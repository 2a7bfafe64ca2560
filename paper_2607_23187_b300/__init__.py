"""B300-native preconditioned Jacobi eigensolver with perturbation-inspired
(spectral-gap-weighted) pivoting (Shao & Nakatsukasa).

The solver lives in the CUDA library ``lib/libpjac.so`` (C ABI declared in
``include/pjac.h``); ``pjac`` is its Python binding.
"""
from . import pjac  # noqa: F401
from .pjac import (Handle, Server, PjacError, pjac_precondition, pjac_solve,  # noqa: F401
                   pjac_solve_batched, pjac_solve_preconditioned, batched_results)

__all__ = ["pjac", "Handle", "Server", "PjacError", "pjac_precondition", "pjac_solve",
           "pjac_solve_preconditioned", "pjac_solve_batched", "batched_results"]
