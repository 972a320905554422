"""Eigenvalue counts and closed-form spectra (oracle; test infrastructure).

The problem (Eq. (1), Section 1) asks for all eigenvalues in (0, gamma].  For
a symmetric-definite pencil, Sylvester's law of inertia gives their number as
the count of negative pivots of an LDL^T factorisation of A - gamma B
(A and B are positive definite, so no eigenvalue is <= 0).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def lambda_1d(n: int, k=None):
    """Eigenvalues of uniform linear FEM on [0,1], n interior nodes, h = 1/(n+1).

    The stiffness stencil (-1, 2, -1)/h and the mass stencil h (1, 4, 1)/6 share
    the eigenvectors sin(k pi i h); their symbols (2 - 2 cos t)/h and
    h (4 + 2 cos t)/6 at t = k pi h give
    lambda_k = (6/h^2) (1 - cos k pi h)/(2 + cos k pi h), k = 1..n, ascending.
    """
    h = 1.0 / (n + 1)
    kk = np.arange(1, n + 1) if k is None else np.asarray(k)
    c = np.cos(kk * np.pi * h)
    return (6.0 / h ** 2) * (1.0 - c) / (2.0 + c)


def eigvec_1d(n: int, k: int):
    """Unnormalised eigenvector sin(k pi i h), i = 1..n, of the 1D pencil."""
    h = 1.0 / (n + 1)
    return np.sin(k * np.pi * h * np.arange(1, n + 1))


def lambda_2d_unit(m: int):
    """Eigenvalues of Q1 FEM with unit coefficient on an m x m grid, Dirichlet.

    The Q1 stiffness is K (x) M + M (x) K and the mass M (x) M with K, M the 1D
    matrices (m-1 interior nodes, h = 1/m), so the eigenvalues are the sums
    lambda_k + lambda_l of the 1D eigenvalues (tensor sum), ascending.
    """
    l1 = lambda_1d(m - 1)
    return np.sort((l1[:, None] + l1[None, :]).ravel())


def sturm_count_tridiag(diag, off, shift_diag=None):
    """Negative pivots of the LDL^T recurrence of a symmetric tridiagonal matrix.

    d_1 = t_11, d_i = t_ii - t_{i,i-1}^2 / d_{i-1}.
    """
    d_prev = None
    neg = 0
    for i in range(len(diag)):
        d = diag[i] if d_prev is None else diag[i] - off[i - 1] ** 2 / d_prev
        if d < 0:
            neg += 1
        d_prev = d
    return neg


def count_below_1d(n: int, gamma: float) -> int:
    """#{lambda <= gamma} for the 1D pencil via the Sturm recurrence on A - gamma B."""
    h = 1.0 / (n + 1)
    diag = np.full(n, 2.0 / h - gamma * 4.0 * h / 6.0)
    off = np.full(n - 1, -1.0 / h - gamma * h / 6.0)
    return sturm_count_tridiag(diag, off)


def count_below_dense(A, B, gamma: float) -> int:
    """#{lambda <= gamma} from the inertia of a dense Bunch-Kaufman LDL^T of A - gamma B."""
    M = (A - gamma * B)
    M = M.toarray() if sp.issparse(M) else np.asarray(M)
    _, D, _ = la.ldl(M)
    # D is block diagonal with 1x1 and 2x2 blocks; its inertia is that of M.
    ev = la.eigvalsh(D)
    return int(np.sum(ev < 0))


def count_below_sparse(A, B, gamma: float) -> int:
    """#{lambda <= gamma} from the pivots of a symmetric sparse LU of A - gamma B.

    SuperLU in symmetric mode with diagonal pivoting only (threshold 0) applies
    the same permutation to rows and columns, so P (A - gamma B) P^T = L U with
    U = D L^T and the signs of diag(U) are the inertia.  The permutations are
    checked to be equal.
    """
    M = (A - gamma * B).tocsc()
    lu = sla.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                  options=dict(SymmetricMode=True))
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("symmetric LU used unequal row/column permutations")
    return int(np.sum(lu.U.diagonal() < 0))


def lowest_eigs(A, B, k: int, dense_limit: int = 3000):
    """The k smallest eigenpairs of (A, B), ascending, B-orthonormal vectors.

    Dense LAPACK (``scipy.linalg.eigh``) up to ``dense_limit``; above it ARPACK
    in shift-invert mode about 0 (``scipy.sparse.linalg.eigsh``).
    """
    n = A.shape[0]
    if n <= dense_limit:
        lam, X = la.eigh(A.toarray() if sp.issparse(A) else A,
                         B.toarray() if sp.issparse(B) else B)
        return lam[:k], X[:, :k]
    # shift-invert about 0: the operator A^{-1} applied through one SuperLU
    # factorisation with a minimum-degree ordering of A + A^T (far less fill
    # than the default column ordering on 3D elasticity)
    lu = sla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
    op = sla.LinearOperator(A.shape, matvec=lu.solve, dtype=float)
    lam, X = sla.eigsh(A.tocsc(), k=k, M=B.tocsc(), sigma=0.0, which="LM", tol=1e-14, OPinv=op)
    order = np.argsort(lam)
    return lam[order], X[:, order]
