"""Rayleigh-Ritz and residual norms (oracle; test infrastructure).

Algorithm 1, after the filter: form A_hat = U^T A U and B_hat = U^T B U,
solve A_hat s_i = theta_i B_hat s_i with theta ascending, set x_i = U s_i, and
compute rho_i = ||A x_i - theta_i B x_i||_2 / (|theta_i| ||B x_i||_2).
Eigenvectors are B-normalised, ||x_i||_B = 1 (notation paragraph of Section 1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la


def rayleigh_ritz(A, B, U):
    """Ritz values (ascending) and B-orthonormal Ritz vectors of span(U).

    The columns of U are first scaled to unit B-norm.  That is a diagonal
    congruence of (A_hat, B_hat), so it changes neither the Ritz values nor the
    Ritz vectors; it only keeps the Cholesky factorisation inside the dense
    generalized eigensolver well scaled when the filtered columns are graded.
    """
    BU = B @ U
    AU = A @ U
    scale = 1.0 / np.sqrt(np.einsum("ij,ij->j", U, BU))
    Us = U * scale[None, :]
    Ah = (Us.T @ (AU * scale[None, :]))
    Bh = (Us.T @ (BU * scale[None, :]))
    Ah = 0.5 * (Ah + Ah.T)
    Bh = 0.5 * (Bh + Bh.T)
    theta, S = la.eigh(Ah, Bh)
    X = Us @ S
    return theta, X


def residuals(A, B, X, theta):
    """rho_i of Algorithm 1 and the variant ||A x - theta B x|| / ||A x||."""
    AX = A @ X
    BX = B @ X
    R = AX - BX * theta[None, :]
    nr = np.linalg.norm(R, axis=0)
    rho = nr / (np.abs(theta) * np.linalg.norm(BX, axis=0))
    rho_ax = nr / np.linalg.norm(AX, axis=0)
    return rho, rho_ax
