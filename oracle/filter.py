"""The rational filter operator with exact shifted solves (oracle; test infrastructure).

Section 3: with quadrature nodes sigma_j and weights w_j, the filter applied to
a block is Phi(A, B) V = sum_{j=1}^{2N} w_j (A - sigma_j B)^{-1} B V.  Since A
and B are real and the nodes come in conjugate pairs (sigma_{N+j} =
conj(sigma_j), w_{N+j} = conj(w_j)), the two members of a pair sum to
2 Re(w_j (A - sigma_j B)^{-1} B V), so only the N upper-half systems are
solved (Algorithm 1, the solve loop and the accumulation U = sum 2 Re(w_j Y_j)).

Shifted systems are solved exactly by sparse LU (SuperLU), the direct method
the paper cites for Eq. (2) in Section 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def shifted_lu(A: sp.spmatrix, B: sp.spmatrix, sigma: complex):
    """Sparse LU of the complex matrix A - sigma B (Eq. (2))."""
    C = (A.astype(complex) - sigma * B.astype(complex)).tocsc()
    return sla.splu(C)


def shifted_solve(A, B, sigma, F):
    """Y = (A - sigma B)^{-1} F for a block F (Eq. (2))."""
    return shifted_lu(A, B, sigma).solve(np.asarray(F, dtype=complex))


def filter_apply(A, B, sigma, w, V):
    """U = sum_j 2 Re(w_j (A - sigma_j B)^{-1} B V) (Algorithm 1, solve + accumulate)."""
    F = B @ V
    U = np.zeros(V.shape, dtype=float)
    for s, wj in zip(np.atleast_1d(sigma), np.atleast_1d(w)):
        Y = shifted_solve(A, B, s, F)
        U += 2.0 * np.real(wj * Y)
    return U


def filter_apply_corrected(A, B, sigma, w, X, theta):
    """The same operator written around a Ritz pair (X, Theta).

    For any X and real diagonal Theta, multiplying through by (A - sigma B)
    shows (A - sigma B)^{-1} B X = X D + (A - sigma B)^{-1} R D with
    R = B X Theta - A X and D = (Theta - sigma I)^{-1}.  Summing the pole terms,

        Phi(A, B) X = X Phi(Theta) + sum_j 2 Re(w_j (A - sigma_j B)^{-1} R D_j).

    This is an identity, so with exact solves it equals ``filter_apply(X)``.
    """
    theta = np.asarray(theta, dtype=float)
    R = (B @ X) * theta[None, :] - A @ X
    phi_theta = np.zeros_like(theta)
    U = np.zeros(X.shape, dtype=float)
    for s, wj in zip(np.atleast_1d(sigma), np.atleast_1d(w)):
        d = 1.0 / (theta - s)
        phi_theta += 2.0 * np.real(wj * d)
        Z = shifted_solve(A, B, s, R)
        U += 2.0 * np.real(wj * Z * d[None, :])
    return X * phi_theta[None, :] + U


def shifted_product(A, B, sigma, P):
    """Q = (A - sigma B) P for a complex block P: the operator of Eq. (2)."""
    P = np.asarray(P, dtype=complex)
    return (A @ P.real + 1j * (A @ P.imag)) - sigma * (B @ P.real + 1j * (B @ P.imag))
