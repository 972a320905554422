"""Finite-element vibration pencils (A = stiffness, B = consistent mass).

The paper's test pencils come from FreeFEM++ models that are not published
(Section 4.1): a 2D beam (P1 triangles), a 3D hollow platform (P2 tetrahedra)
and a 3D fish-like body (P1 tetrahedra), all linear elasticity with one part of
the boundary fixed.  These generators stand in for them with pencils of the
same character on structured grids:

* ``pencil_1d``          -- linear elements on [0, 1], Dirichlet ends.
* ``pencil_2d_q1``       -- bilinear elements on [0, 1]^2, Dirichlet boundary,
                            lognormal coefficient per element.
* ``pencil_3d_elasticity`` -- trilinear hexahedra on [0, 1]^3, isotropic linear
                            elasticity, lognormal Young's modulus per element,
                            face x = 0 clamped.

A and B always share one sparsity pattern (the union pattern, explicit zeros
kept), are real symmetric, and are positive definite once the Dirichlet degrees
of freedom are eliminated.  Element matrices are integrated with the 2-point
Gauss rule per direction, which is exact for both the stiffness and the mass
of (bi/tri)linear elements on a uniform grid.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

BASE_SEED = 2503


@dataclasses.dataclass
class Pencil:
    """A sparse symmetric-definite pencil in CSR form on one shared pattern."""
    n: int
    row_ptr: np.ndarray   # int32, n + 1
    col_idx: np.ndarray   # int32, nnz, sorted within each row
    a_val: np.ndarray     # float64, nnz (stiffness)
    b_val: np.ndarray     # float64, nnz (mass)
    kind: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def A(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.a_val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def B(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.b_val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _assemble(n, rows, cols, avals, bvals, kind, meta) -> Pencil:
    """Sum COO triplets of A and B into CSR on their common (union) pattern."""
    keep = (rows >= 0) & (cols >= 0)
    rows = rows[keep].astype(np.int64)
    cols = cols[keep].astype(np.int64)
    avals = avals[keep]
    bvals = bvals[keep]
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    uniq_start = np.flatnonzero(np.concatenate(([True], key[1:] != key[:-1])))
    ukey = key[uniq_start]
    a = np.add.reduceat(avals[order], uniq_start)
    b = np.add.reduceat(bvals[order], uniq_start)
    r = (ukey // n).astype(np.int64)
    c = (ukey % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    if row_ptr[-1] >= 2**31:
        raise ValueError("pattern too large for 32-bit indices")
    return Pencil(n=n, row_ptr=row_ptr.astype(np.int32), col_idx=c,
                  a_val=np.ascontiguousarray(a, dtype=np.float64),
                  b_val=np.ascontiguousarray(b, dtype=np.float64), kind=kind, meta=meta)


# --------------------------------------------------------------------------
# 1D linear elements
# --------------------------------------------------------------------------
def pencil_1d(n: int) -> Pencil:
    """Uniform linear FEM on [0, 1] with n interior nodes (h = 1/(n+1)).

    A = tridiag(-1, 2, -1)/h, B = h*tridiag(1, 4, 1)/6.
    """
    h = 1.0 / (n + 1)
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    av = np.concatenate([np.full(n, 2.0 / h), np.full(n - 1, -1.0 / h), np.full(n - 1, -1.0 / h)])
    bv = np.concatenate([np.full(n, 4.0 * h / 6.0), np.full(n - 1, h / 6.0), np.full(n - 1, h / 6.0)])
    return _assemble(n, rows, cols, av, bv, "1d", {"h": h})


# --------------------------------------------------------------------------
# reference elements by Gauss quadrature
# --------------------------------------------------------------------------
_GP = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
_GW = np.array([0.5, 0.5])


def _shape_1d(x):
    """Linear shape functions on [0,1] and their derivatives (node 0 at 0)."""
    return np.array([1.0 - x, x]), np.array([-1.0, 1.0])


def q1_element(h: float):
    """Unit-coefficient Laplace stiffness and mass of a square bilinear element.

    Local node (a, b) -> index a + 2 b, with a the x offset and b the y offset.
    """
    K = np.zeros((4, 4))
    M = np.zeros((4, 4))
    for gx, wx in zip(_GP, _GW):
        for gy, wy in zip(_GP, _GW):
            Nx, dNx = _shape_1d(gx)
            Ny, dNy = _shape_1d(gy)
            N = np.array([Nx[a] * Ny[b] for b in range(2) for a in range(2)])
            dx = np.array([dNx[a] * Ny[b] for b in range(2) for a in range(2)]) / h
            dy = np.array([Nx[a] * dNy[b] for b in range(2) for a in range(2)]) / h
            w = wx * wy * h * h
            K += w * (np.outer(dx, dx) + np.outer(dy, dy))
            M += w * np.outer(N, N)
    return 0.5 * (K + K.T), 0.5 * (M + M.T)


def hex8_elasticity_element(h: float, nu: float, rho: float = 1.0):
    """Stiffness (Young's modulus 1) and mass of a cubic trilinear element.

    Degrees of freedom are ordered node-major: 3 * (a + 2 b + 4 c) + component.
    Strains use Voigt order (xx, yy, zz, yz, xz, xy) with engineering shears.
    """
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D += np.diag([2 * mu, 2 * mu, 2 * mu, mu, mu, mu])
    K = np.zeros((24, 24))
    M = np.zeros((24, 24))
    for gx, wx in zip(_GP, _GW):
        for gy, wy in zip(_GP, _GW):
            for gz, wz in zip(_GP, _GW):
                Nx, dNx = _shape_1d(gx)
                Ny, dNy = _shape_1d(gy)
                Nz, dNz = _shape_1d(gz)
                idx = [(a, b, c) for c in range(2) for b in range(2) for a in range(2)]
                N = np.array([Nx[a] * Ny[b] * Nz[c] for a, b, c in idx])
                gxv = np.array([dNx[a] * Ny[b] * Nz[c] for a, b, c in idx]) / h
                gyv = np.array([Nx[a] * dNy[b] * Nz[c] for a, b, c in idx]) / h
                gzv = np.array([Nx[a] * Ny[b] * dNz[c] for a, b, c in idx]) / h
                Bm = np.zeros((6, 24))
                for k in range(8):
                    Bm[0, 3 * k + 0] = gxv[k]
                    Bm[1, 3 * k + 1] = gyv[k]
                    Bm[2, 3 * k + 2] = gzv[k]
                    Bm[3, 3 * k + 1] = gzv[k]
                    Bm[3, 3 * k + 2] = gyv[k]
                    Bm[4, 3 * k + 0] = gzv[k]
                    Bm[4, 3 * k + 2] = gxv[k]
                    Bm[5, 3 * k + 0] = gyv[k]
                    Bm[5, 3 * k + 1] = gxv[k]
                w = wx * wy * wz * h ** 3
                K += w * Bm.T @ D @ Bm
                NN = np.outer(N, N)
                for comp in range(3):
                    M[comp::3, comp::3] += w * rho * NN
    return 0.5 * (K + K.T), 0.5 * (M + M.T)


# --------------------------------------------------------------------------
# 2D bilinear, lognormal coefficient
# --------------------------------------------------------------------------
def pencil_2d_q1(m: int, seed: int | None = BASE_SEED + 2, sigma: float = 0.5) -> Pencil:
    """Q1 FEM of -div(c grad u) = lambda u on an m x m grid of [0,1]^2.

    Homogeneous Dirichlet on the whole boundary, so n = (m-1)^2.  The
    coefficient c is constant per element, lognormal(0, sigma) of an underlying
    normal drawn from ``default_rng(seed)`` in x-fastest element order; with
    ``seed=None`` it is identically 1.  The mass is consistent with density 1.
    """
    h = 1.0 / m
    Ke, Me = q1_element(h)
    nelem = m * m
    if seed is None:
        coef = np.ones(nelem)
    else:
        coef = np.random.default_rng(seed).lognormal(mean=0.0, sigma=sigma, size=nelem)
    ex, ey = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ex = ex.ravel()
    ey = ey.ravel()   # element e = ex + m*ey (x fastest)

    def free(ix, iy):
        inside = (ix >= 1) & (ix <= m - 1) & (iy >= 1) & (iy <= m - 1)
        return np.where(inside, (ix - 1) + (m - 1) * (iy - 1), -1)

    dofs = np.stack([free(ex + a, ey + b) for b in range(2) for a in range(2)], axis=1)  # (nelem, 4)
    rows = np.repeat(dofs, 4, axis=1).ravel()
    cols = np.tile(dofs, (1, 4)).ravel()
    av = (coef[:, None] * Ke.ravel()[None, :]).ravel()
    bv = np.broadcast_to(Me.ravel()[None, :], (nelem, 16)).ravel().copy()
    n = (m - 1) ** 2
    return _assemble(n, rows, cols, av, bv, "2d_q1", {"m": m, "h": h, "seed": seed, "sigma": sigma})


# --------------------------------------------------------------------------
# 3D trilinear elasticity, lognormal Young's modulus, face x=0 clamped
# --------------------------------------------------------------------------
def pencil_3d_elasticity(nodes_per_edge: int, seed: int | None = BASE_SEED + 3,
                         sigma: float = 0.5, nu: float = 0.3, rho: float = 1.0) -> Pencil:
    """Trilinear-hexahedron linear elasticity on the unit cube.

    ``nodes_per_edge`` nodes per edge (h = 1/(nodes_per_edge-1)); the face x = 0
    is clamped and its degrees of freedom eliminated, so
    n = 3 * (p-1) * p * p with p = nodes_per_edge.  Young's modulus is
    lognormal(0, sigma) per element (x-fastest order, ``default_rng(seed)``),
    Poisson ratio ``nu``, density ``rho``.
    """
    p = nodes_per_edge
    ne = p - 1
    h = 1.0 / ne
    Ke, Me = hex8_elasticity_element(h, nu, rho)
    nelem = ne ** 3
    if seed is None:
        E = np.ones(nelem)
    else:
        E = np.random.default_rng(seed).lognormal(mean=0.0, sigma=sigma, size=nelem)
    ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    ex = ex.ravel()
    ey = ey.ravel()
    ez = ez.ravel()   # element e = ex + ne*(ey + ne*ez)

    def free_node(ix, iy, iz):
        return np.where(ix >= 1, (ix - 1) + (p - 1) * (iy + p * iz), -1)

    nodes = np.stack([free_node(ex + a, ey + b, ez + c)
                      for c in range(2) for b in range(2) for a in range(2)], axis=1)  # (nelem, 8)
    dofs = np.where(nodes[:, :, None] >= 0, 3 * nodes[:, :, None] + np.arange(3)[None, None, :], -1)
    dofs = dofs.reshape(nelem, 24)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    av = (E[:, None] * Ke.ravel()[None, :]).ravel()
    bv = np.broadcast_to(Me.ravel()[None, :], (nelem, 576)).ravel().copy()
    n = 3 * (p - 1) * p * p
    return _assemble(n, rows, cols, av, bv, "3d_elasticity",
                     {"p": p, "h": h, "seed": seed, "sigma": sigma, "nu": nu, "rho": rho})


def rigid_body_modes(pencil: Pencil) -> np.ndarray:
    """The six rigid-body displacement fields of a ``pencil_3d_elasticity``
    mesh restricted to its free dofs (n x 6, row-major float64): translations
    along x, y, z and rotations about axes through the cube's centre
    (x, y, z) -> (0, -z, y), (z, 0, -x), (-y, x, 0).  They are the near-null
    space of the stiffness away from the clamped face."""
    p = int(pencil.meta["p"])
    h = float(pencil.meta["h"])
    node = np.arange(pencil.n // 3)
    ix = node % (p - 1) + 1
    rest = node // (p - 1)
    iy = rest % p
    iz = rest // p
    x, y, z = ix * h - 0.5, iy * h - 0.5, iz * h - 0.5
    B = np.zeros((pencil.n, 6))
    for c in range(3):
        B[c::3, c] = 1.0
    B[1::3, 3], B[2::3, 3] = -z, y
    B[0::3, 4], B[2::3, 4] = z, -x
    B[0::3, 5], B[1::3, 5] = -y, x
    return np.ascontiguousarray(B)


# --------------------------------------------------------------------------
# start blocks and the named configurations
# --------------------------------------------------------------------------
def start_block(n: int, L: int, seed: int) -> np.ndarray:
    """Seeded standard-normal start block V1 (n x L, row-major float64)."""
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal((n, L)))


# Named workloads.  ``nev`` eigenvalues lie in (0, gamma]; ``L`` is the
# subspace size; ``n_poles`` counts the upper-half-plane poles N (2N poles in
# all, conjugates implied).
CONFIGS = {
    "fem1d_n2000": dict(kind="1d", n=2000, nev=20, L=30, n_poles=2, seed=BASE_SEED + 1),
    "fem2d_q1_300": dict(kind="2d", m=300, nev=100, L=150, n_poles=4, seed=BASE_SEED + 2),
    "fem3d_elastic_40": dict(kind="3d", p=40, nev=200, L=300, n_poles=4, seed=BASE_SEED + 3),
}


def config_pencil(name: str) -> Pencil:
    c = CONFIGS[name]
    if c["kind"] == "1d":
        return pencil_1d(c["n"])
    if c["kind"] == "2d":
        return pencil_2d_q1(c["m"], seed=c["seed"])
    if c["kind"] == "3d":
        return pencil_3d_elasticity(c["p"], seed=c["seed"])
    raise KeyError(name)


def interval_for(name: str) -> dict:
    """The stored interval (0, gamma] for a named workload.

    The values are written by ``tests/golden/make_intervals.py`` (which uses
    only the FP64 oracle) into ``tests/golden/intervals.json``.
    """
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "tests", "golden", "intervals.json")
    with open(path) as f:
        table = json.load(f)
    return table[name]


# --------------------------------------------------------------------------
# problem streams for the batched and serving workloads
# --------------------------------------------------------------------------
def weyl_gamma(kind: str, nev: int) -> float:
    """An interval end expected to hold about ``nev`` eigenvalues.

    Weyl-law estimates of the counting function N(lambda) of the continuous
    problems (geometric-mean coefficient 1): 1D Dirichlet N = sqrt(lambda)/pi;
    2D Dirichlet unit square N = lambda/(4 pi) - sqrt(lambda)/pi; 3D elasticity
    by an empirical fit (below).  The exact count of a discrete pencil differs
    by a few per cent; callers size the subspace with slack.
    """
    k = nev + 0.5
    if kind == "1d":
        return (math.pi * k) ** 2
    if kind == "2d":
        s = 2.0 + math.sqrt(4.0 + 4.0 * math.pi * k)
        return s * s
    if kind == "3d":
        # Weyl's leading term undercounts the clamped cube with free faces (its
        # surface modes); N(lambda) = 0.092 lambda^{3/2} + 0.99 lambda, fitted to
        # dense spectra of these pencils, is solved for lambda by bisection.
        lo, hi = 0.0, 1e6
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if 0.092 * mid ** 1.5 + 0.99 * mid < k:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)
    raise KeyError(kind)


# Largest 1D pencil drawn for a batch.  On [0, 1] with n interior nodes an
# eigenvector stored in FP64 carries rounding noise of relative size eps per
# entry, which the stiffness stencil amplifies by ~sqrt(6)/h while A x itself
# is ~lambda h |x|: the relative residual |A x - lambda B x| / |A x| of the
# lowest pair cannot go below ~sqrt(6) eps n^2 / lambda_1 (lambda_1 ~ pi^2).
# Ritz vectors formed from a basis of L vectors sit about ten times above
# that: measured 1.2e-8 to 1.5e-8 at n = 4 300 .. 4 900, where the 1e-8 gate
# then stagnates.  1D batch members stay at or below 3 000 (floor ~5e-9).
N_MAX_1D = 3000


def random_problem(rng, kind: str, n_lo: int, n_hi: int, nev_lo: int, nev_hi: int, seed: int):
    """One random pencil of the given kind with n log-uniform in [n_lo, n_hi]
    (for 1D in [n_lo, min(n_hi, N_MAX_1D)]).

    Returns dict(pencil, kind, nev_target, L, gamma, V0).  L = 1.5 NEV
    (rounded up to even).  The grid size is rounded to the nearest valid one.
    """
    hi = min(n_hi, max(n_lo, N_MAX_1D)) if kind == "1d" else n_hi
    n_target = math.exp(rng.uniform(math.log(n_lo), math.log(hi)))
    nev = int(rng.integers(nev_lo, nev_hi + 1))
    if kind == "1d":
        pencil = pencil_1d(max(50, int(round(n_target))))
    elif kind == "2d":
        m = max(8, int(round(math.sqrt(n_target)) + 1))
        pencil = pencil_2d_q1(m, seed=seed)
    else:
        p = max(4, int(round((n_target / 3.0) ** (1.0 / 3.0))))
        pencil = pencil_3d_elasticity(p, seed=seed)
    L = int(math.ceil(1.5 * nev / 2.0) * 2)
    L = min(L, pencil.n // 2)
    return dict(pencil=pencil, kind=kind, nev_target=nev, L=L, gamma=weyl_gamma(kind, nev),
                V0=start_block(pencil.n, L, seed + 7))


def batch_workload(count: int = 64, seed: int = BASE_SEED + 4, n_lo: int = 1000, n_hi: int = 50000):
    """Independent pencils: kind uniform in {1d, 2d, 3d}, n log-uniform, NEV in [10, 60]."""
    rng = np.random.default_rng(seed)
    kinds = ("1d", "2d", "3d")
    return [random_problem(rng, kinds[int(rng.integers(0, 3))], n_lo, n_hi, 10, 60, seed * 1000 + i)
            for i in range(count)]


def serving_stream(count: int, seed: int = BASE_SEED + 5, n_lo: int = 10000, n_hi: int = 500000,
                   nev_lo: int = 20, nev_hi: int = 200, rate_per_s: float = 1.0):
    """A Poisson-arrival request stream of 2D/3D pencils (50/50).

    Returns a list of (arrival_time_s, problem dict) sorted by arrival time.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        kind = "2d" if rng.uniform() < 0.5 else "3d"
        out.append((t, random_problem(rng, kind, n_lo, n_hi, nev_lo, nev_hi, seed * 1000 + i)))
    return out
