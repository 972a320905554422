"""Algorithm 1 (rational filter subspace iteration) with exact solves (oracle).

Each outer step k: solve Y_j = (A - sigma_j B)^{-1} B V_k for j = 1..N; form
U = sum_j 2 Re(w_j Y_j); Rayleigh-Ritz on span(U); residuals rho_i; restart
with V_{k+1} = X.  Stopping rule (Section 3, text before Algorithm 1, and
Section 4.2.1): every Ritz pair whose value lies in the wanted interval
(0, gamma] has rho_i <= tau.  Ritz pairs outside the interval are guard vectors
and are not tested (the paper's "i = 1..L" would include them although L
exceeds the number of wanted eigenvalues; the reading here tests the wanted
ones only).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .filter import filter_apply
from .rr import rayleigh_ritz, residuals


@dataclasses.dataclass
class SubspaceResult:
    theta: np.ndarray       # all L Ritz values, ascending
    X: np.ndarray           # n x L, B-orthonormal
    rho: np.ndarray         # residuals rho_i
    rho_ax: np.ndarray      # ||A x - theta B x|| / ||A x||
    n_wanted: int           # Ritz values in (0, gamma]
    iters: int
    converged: bool
    history: list


def subspace_iterate(A, B, sigma, w, gamma, V1, tol=1e-12, max_outer=50, min_outer=1,
                     floor_stop=1e-8):
    """Run Algorithm 1 from V1 until the wanted Ritz pairs reach ``tol``.

    The attainable rho is bounded below by rounding, about eps * lambda_max /
    lambda_i, which for FE pencils can exceed a very small ``tol``.  Once the
    worst wanted residual is below ``floor_stop`` and stops decreasing (it
    falls by less than a factor 2 in one step), the iteration has reached that
    floor and stops as converged.
    """
    V = np.array(V1, dtype=float, copy=True)
    history = []
    theta = X = rho = rho_ax = None
    for k in range(1, max_outer + 1):
        U = filter_apply(A, B, sigma, w, V)
        theta, X = rayleigh_ritz(A, B, U)
        rho, rho_ax = residuals(A, B, X, theta)
        wanted = (theta > 0) & (theta <= gamma)
        worst = float(np.max(rho[wanted])) if wanted.any() else np.inf
        history.append(worst)
        V = X
        stalled = len(history) >= 2 and worst <= floor_stop and worst > 0.5 * history[-2]
        if k >= min_outer and wanted.any() and (worst <= tol or stalled):
            return SubspaceResult(theta, X, rho, rho_ax, int(wanted.sum()), k, True, history)
    wanted = (theta > 0) & (theta <= gamma)
    return SubspaceResult(theta, X, rho, rho_ax, int(wanted.sum()), max_outer, False, history)
