"""GB300 (sm_103a) shifted Laplace rational-filter eigensolver.

Finds all eigenpairs of a sparse symmetric-definite pencil A x = lambda B x in
(0, gamma] by rational-filter subspace iteration: the filter
sum_j 2 Re(w_j (A - sigma_j B)^{-1} B) is applied to a block by batched
preconditioned COCG over all poles and columns, followed by Cholesky-QR2
B-orthonormalisation and Rayleigh-Ritz.  The compute lives in the CUDA library
``libslrf.so`` (C ABI in ``include/slrf.h``); this package is its binding.
"""
from .api import (Filter, Handle, SlrfError, default_opts, design_poles, filter_eval, load,  # noqa: F401
                  mg_describe, mg_transfer, OK, NOT_CONVERGED, SUBSPACE_TOO_SMALL, CHOLQR_FAIL, PREC_FP64, PREC_MIXED,
                  PRECOND_NONE, PRECOND_JACOBI, PRECOND_MG, PRECOND_AUTO)

__all__ = ["Filter", "Handle", "SlrfError", "default_opts", "design_poles", "filter_eval", "load", "mg_describe",
           "mg_transfer"]
