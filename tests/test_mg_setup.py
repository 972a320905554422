"""CPU checks of the multigrid hierarchy the library builds on the host for the
SLRF_PRECOND_MG preconditioner (slrf_mg_describe; no GPU).

The coarsest pencil is a Galerkin projection (P^T A P, P^T B P) of the input
pencil onto range(P), so its eigenvalues are Ritz values of (A, B): by the
Courant-Fischer theorem theta_k >= lambda_k and theta_max <= lambda_max.  Its
eigenvalues, computed by the library's own Householder + implicit QR solver,
are compared with LAPACK on the returned dense coarse pencil."""
import ctypes as C

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import inertia
from workloads import config_pencil, interval_for, pencil_1d, pencil_2d_q1, pencil_3d_elasticity


@pytest.fixture(scope="module")
def api(lib):
    from paper_2503_21618_gb300 import api as a
    return a


def test_levels_shrink_to_the_coarse_target(api):
    d = api.mg_describe(pencil_1d(2000))
    lv = d["levels"]
    assert lv[0] == 2000 and lv[-1] <= 256
    assert all(b <= a / 2 for a, b in zip(lv, lv[1:]))
    d2 = api.mg_describe(pencil_1d(2000), api.default_opts(mg_coarse=40))
    assert d2["levels"][-1] <= 40 and len(d2["levels"]) > len(lv)


@pytest.mark.parametrize("name", ["fem1d_n2000", "fem2d_q1_300"])
def test_coarse_eigensolver_matches_lapack(api, name):
    d = api.mg_describe(config_pencil(name), coarse=True)
    Ac, Bc, lam = d["coarse_A"], d["coarse_B"], d["coarse_lambda"]
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-12 * np.abs(Ac).max())
    assert np.allclose(Bc, Bc.T, rtol=0, atol=1e-12 * np.abs(Bc).max())
    ref = sla.eigh(Ac, Bc, eigvals_only=True)
    assert np.all(np.diff(lam) >= 0)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)


def test_large_coarse_level_eigensolver_matches_lapack(api):
    # a 725-unknown coarsest level: the size at which the solve of a deep
    # shift stops the cycle; the eigensolver runs on several threads there
    p = pencil_2d_q1(80, seed=7)
    o = api.default_opts(mg_coarse=800)
    d = api.mg_describe(p, o, coarse=True)
    assert d["levels"] == [6241, 725]
    ref = sla.eigh(d["coarse_A"], d["coarse_B"], eigvals_only=True)
    np.testing.assert_allclose(d["coarse_lambda"], ref, rtol=1e-10)


def test_coarse_ritz_values_bound_the_1d_spectrum(api):
    n = 2000
    d = api.mg_describe(pencil_1d(n), coarse=True)
    lam = d["coarse_lambda"]
    exact = inertia.lambda_1d(n)            # closed form, ascending
    k = len(lam)
    assert np.all(lam >= exact[:k] * (1 - 1e-12))
    assert lam[-1] <= exact[-1] * (1 + 1e-12)
    # smoothed aggregation keeps the smooth modes: the lowest Ritz values are close
    assert lam[0] <= exact[0] * 1.01 and lam[4] <= exact[4] * 1.05


def test_coarse_ritz_values_bound_the_2d_spectrum(api):
    name = "fem2d_q1_300"
    d = api.mg_describe(config_pencil(name), coarse=True)
    lam = d["coarse_lambda"]
    ref = np.array(interval_for(name)["lambda"])
    k = min(len(ref), len(lam))
    assert np.all(lam[:k] >= ref[:k] * (1 - 1e-12))
    assert lam[0] <= 2.0 * ref[0]


def test_single_level_is_the_pencil_itself(api):
    n = 200
    p = pencil_1d(n)
    d = api.mg_describe(p, coarse=True)
    assert d["levels"] == [n]
    np.testing.assert_array_equal(d["coarse_A"], p.A().toarray())
    np.testing.assert_array_equal(d["coarse_B"], p.B().toarray())
    np.testing.assert_allclose(d["coarse_lambda"], inertia.lambda_1d(n), rtol=1e-10)


def test_node_blocks_are_kept_on_every_level(api):
    p = pencil_3d_elasticity(6)
    d = api.mg_describe(p, api.default_opts(mg_coarse=30))
    assert len(d["levels"]) >= 2
    assert all(n % 3 == 0 for n in d["levels"])
    d1 = api.mg_describe(p, api.default_opts(mg_coarse=30, mg_block=1))
    assert d1["levels"] != d["levels"]


def test_setup_is_deterministic(api):
    p = pencil_2d_q1(60)
    a = api.mg_describe(p, coarse=True)
    b = api.mg_describe(p, coarse=True)
    assert a["levels"] == b["levels"] and a["nnz"] == b["nnz"]
    assert np.array_equal(a["coarse_lambda"], b["coarse_lambda"])
    assert np.array_equal(a["coarse_A"], b["coarse_A"])


def test_describe_rejects_bad_input(api, lib):
    p = pencil_1d(50)
    keep = [np.ascontiguousarray(p.row_ptr, dtype=np.int32), np.ascontiguousarray(p.col_idx, dtype=np.int32),
            np.ascontiguousarray(p.a_val, dtype=np.float64), np.ascontiguousarray(p.b_val, dtype=np.float64)]
    nl = C.c_int32()
    ln = (C.c_int64 * api.MG_MAX_LEVELS)()
    lz = (C.c_int64 * api.MG_MAX_LEVELS)()
    o = api.default_opts()
    dev = api.slrf_pencil(p.n, keep[1].size, *[a.ctypes.data for a in keep], 1)
    assert lib.slrf_mg_describe(C.byref(dev), C.byref(o), C.byref(nl), ln, lz, None, None, None, None) == api.EINVAL
    bad = keep[2].copy()
    bad[0] = -1.0                                   # non-positive diagonal
    hb = api.slrf_pencil(p.n, keep[1].size, keep[0].ctypes.data, keep[1].ctypes.data, bad.ctypes.data,
                         keep[3].ctypes.data, 0)
    assert lib.slrf_mg_describe(C.byref(hb), C.byref(o), C.byref(nl), ln, lz, None, None, None, None) == api.EINVAL
    o.mg_omega = 2.5
    ok = api.slrf_pencil(p.n, keep[1].size, *[a.ctypes.data for a in keep], 0)
    assert lib.slrf_mg_describe(C.byref(ok), C.byref(o), C.byref(nl), ln, lz, None, None, None, None) == api.EINVAL


def _prolongators(api, p, o):
    import scipy.sparse as sp
    Ps, rhos = [], []
    for l in range(len(api.mg_describe(p, o)["levels"]) - 1):
        (ptr, col, val, nr, nc), rho = api.mg_transfer(p, l, o)
        Ps.append(sp.csr_matrix((val, col, ptr), shape=(nr, nc)))
        rhos.append(rho)
    return Ps, rhos


@pytest.mark.parametrize("pencil,opts", [(lambda: pencil_2d_q1(22, seed=9), dict(mg_coarse=16)),
                                         (lambda: pencil_1d(2000), dict()),
                                         (lambda: pencil_3d_elasticity(5), dict(mg_coarse=30))])
def test_prolongators_reproduce_the_galerkin_coarse_pencil(api, pencil, opts):
    # P_l^T A_l P_l chained from the exported prolongators (scipy) must give the
    # coarsest pencil the library formed itself; rho_l must be the spectral
    # radius of diag(A_l)^{-1} A_l to within the few percent that its 30
    # power-iteration steps reach (the damping omega / rho_l needs no more)
    p = pencil()
    o = api.default_opts(**opts)
    d = api.mg_describe(p, o, coarse=True)
    Ps, rhos = _prolongators(api, p, o)
    A, B = p.A().tocsr(), p.B().tocsr()
    for l, P in enumerate(Ps):
        assert P.shape == (d["levels"][l], d["levels"][l + 1])
        Dinv_A = (A.multiply(1.0 / A.diagonal()[:, None])).toarray()
        lam_max = np.max(np.abs(np.linalg.eigvals(Dinv_A))) if A.shape[0] <= 2000 else None
        if lam_max is not None:
            assert abs(rhos[l] - lam_max) <= 0.05 * lam_max
        A, B = (P.T @ A @ P).tocsr(), (P.T @ B @ P).tocsr()
    scale = np.abs(d["coarse_A"]).max()
    np.testing.assert_allclose(A.toarray(), d["coarse_A"], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(B.toarray(), d["coarse_B"], rtol=0, atol=1e-12 * np.abs(d["coarse_B"]).max())


def test_prolongator_is_a_smoothed_piecewise_constant(api):
    # P = (I - 4/(3 rho) diag(A)^{-1} A) T with T piecewise constant on the
    # aggregates (T 1 = 1/sqrt(|aggregate|) per row).  In 1D the aggregates
    # are a node and its two strong neighbours (n = 300 -> 100 aggregates;
    # the first and the last differ), so T 1 = 1/sqrt(3) and A T 1 = 0 a few
    # nodes away from the ends: P 1 = T 1 there
    p = pencil_1d(300)
    (ptr, col, val, nr, nc), rho = api.mg_transfer(p, 0)
    import scipy.sparse as sp
    P = sp.csr_matrix((val, col, ptr), shape=(nr, nc))
    assert nc == 100
    rows = np.asarray(P.sum(axis=1)).ravel()
    np.testing.assert_allclose(rows[4:-6], 1 / np.sqrt(3), rtol=1e-13)
    assert np.all(np.diff(P.indptr) <= 2)           # a node touches at most two aggregates


def test_fused_finest_level_equals_the_two_grid_steps(api):
    # The cycle's finest level restricts and prolongs through F = (M - D^{-1}) P:
    # r1 = -F^T (D r) and z = D (2 r - M (D r) - F e) are the textbook steps
    # x = D r, r1 = P^T (r - M x), z1 = x + P e, z = z1 + D (r - M z1)
    import scipy.sparse as sp
    from oracle import poles
    p = pencil_2d_q1(22, seed=9)
    o = api.default_opts(mg_coarse=16)
    Ps, rhos = _prolongators(api, p, o)
    P = Ps[0]
    A, B = p.A().tocsr(), p.B().tocsr()
    s, _ = poles.slrf_poles(4, 1.0, 0.01, 3000.0)
    rng = np.random.default_rng(1)
    for sig in s:
        M = (A - sig * B).tocsr()
        Dd = (o.mg_omega / rhos[0]) / (A.diagonal() - sig * B.diagonal())
        D = sp.diags(Dd)
        Mc = (P.T @ M @ P).toarray()
        r = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
        x = D @ r
        r1 = P.T @ (r - M @ x)
        e = np.linalg.solve(Mc, r1)
        z1 = x + P @ e
        z = z1 + D @ (r - M @ z1)
        F = (M - sp.diags(1.0 / Dd)) @ P
        r1f = -(F.T @ (D @ r))
        zf = D @ (2 * r - M @ (D @ r) - F @ np.linalg.solve(Mc, r1f))
        assert np.linalg.norm(r1f - r1) <= 1e-13 * np.linalg.norm(r1)
        assert np.linalg.norm(zf - z) <= 1e-13 * np.linalg.norm(z)


def test_transfer_rejects_bad_levels(api):
    p = pencil_2d_q1(22, seed=9)
    o = api.default_opts(mg_coarse=16)
    nlev = len(api.mg_describe(p, o)["levels"])
    with pytest.raises(api.SlrfError):
        api.mg_transfer(p, nlev - 1, o)
    with pytest.raises(api.SlrfError):
        api.mg_transfer(p, -1, o)
