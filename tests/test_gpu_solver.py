"""GPU parity of the filter and of Algorithm 1 against the FP64 oracle,
through the C ABI, from small cases up to the full benchmark workload."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as la

from oracle import filter as ofilt
from oracle import inertia, poles
from workloads import config_pencil, interval_for, pencil_1d, pencil_2d_q1, pencil_3d_elasticity, start_block

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21618_gb300 import api as a
    return a


def rel_err(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# --------------------------------------------------------------------------
# filter operator (Section 3; Algorithm 1 solve + accumulate)
# --------------------------------------------------------------------------
# N = 9 exercises the 16-pole register path of the update kernel; it uses the
# Gauss-Legendre rule because the SLRF design with N > 8 has weights ~1e6 whose
# cancellation in the pole sum limits any filter to ~1e-6 relative accuracy.
@pytest.mark.parametrize("rule,N", [("gauss_legendre", 4), ("midpoint", 3), ("slrf", 4), ("gauss_legendre", 9)])
def test_filter_apply_fp64_matches_exact_lu(api, rule, N):
    p = pencil_2d_q1(22, seed=9)           # n = 441
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[14] + lam[15])
    s, w = (poles.slrf_poles(N, 1.0, 0.01, gamma) if rule == "slrf" else poles.quadrature_poles(rule, N, gamma))
    V = start_block(p.n, 19, 4)
    h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=2000))
    U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    Uo = ofilt.filter_apply(p.A(), p.B(), s, w, V)
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), Uo) < 1e-10
    assert rep.spmv > 0 and rep.kernel_launches > 0


def test_filter_apply_mixed_fp32(api):
    p = pencil_2d_q1(30, seed=1)
    gamma = 800.0
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    V = start_block(p.n, 12, 5)
    h = api.Handle(p, api.default_opts(precision=api.PREC_MIXED, inner_tol=1e-5))
    U, st, _ = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    Uo = ofilt.filter_apply(p.A(), p.B(), s, w, V)
    # A single FP32 filter application is accurate to about kappa(A - sigma B)
    # times its relative residual (here ~1e-3); the subspace iteration recovers
    # FP64 accuracy through the residual-corrected filter (tests below).
    assert rel_err(U.cpu().numpy(), Uo) < 2e-2


def test_filter_on_exact_eigenvectors_is_phi(api):
    # Phi(A, B) x_k = Phi(lambda_k) x_k for the closed-form 1D eigenvectors
    n = 200
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[7] + lam[8])
    s, w = poles.quadrature_poles("gauss_legendre", 4, gamma)
    ks = [1, 3, 8, 9, 20]
    V = np.stack([inertia.eigvec_1d(n, k) for k in ks], axis=1)
    h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=5000))
    U, st, _ = h.filter_apply(api.Filter(s, w), torch.from_numpy(np.ascontiguousarray(V)).cuda())
    phi = poles.phi_real(lam[np.array(ks) - 1], s, w)
    np.testing.assert_allclose(U.cpu().numpy(), V * phi[None, :], atol=1e-9)


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
def _check_eigs(theta, resid, lam_ref, nev, tol_eig=1e-10):
    wanted = theta[:nev]
    np.testing.assert_allclose(wanted, lam_ref[:nev], rtol=tol_eig)
    assert resid[:nev].max() <= 1e-8


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_subspace_1d_config(api, prec):
    name = "fem1d_n2000"
    p = config_pencil(name)
    iv = interval_for(name)
    lam = inertia.lambda_1d(p.n)
    s, w = poles.slrf_poles(2, 1.0, 0.01, iv["gamma"])
    V0 = start_block(p.n, iv["L"], 2504)
    opts = (api.default_opts() if prec == "mixed"
            else api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=1000))
    h = api.Handle(p, opts)
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), iv["gamma"], torch.from_numpy(V0).cuda(),
                                                         tol=1e-8, max_outer=40)
    theta = theta.cpu().numpy()
    resid = resid.cpu().numpy()
    assert st == api.OK, (st, rep.outer_iters, rep.max_resid)
    assert nconv == 20 == rep.n_wanted == inertia.count_below_1d(p.n, iv["gamma"])
    _check_eigs(theta, resid, lam, 20)
    assert rep.max_resid_ax <= 1e-8
    Xh = X.cpu().numpy()
    np.testing.assert_allclose(Xh[:, :20].T @ (p.B() @ Xh[:, :20]), np.eye(20), atol=1e-10)


@pytest.mark.parametrize("kernel", [0, 1, 2, 4])
def test_subspace_2d_small_matches_dense(api, kernel):
    # shifted product kernel 0 = autotuned, 1 = row groups, 2 = staged, 4 = SELL-C-sigma
    p = pencil_2d_q1(40, seed=21)          # n = 1521
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    nev = 30
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    V0 = start_block(p.n, 45, 7)
    h = api.Handle(p, api.default_opts(spmm_kernel=kernel))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma, torch.from_numpy(V0).cuda())
    assert st == api.OK and nconv == nev == inertia.count_below_sparse(p.A(), p.B(), gamma)
    _check_eigs(theta.cpu().numpy(), resid.cpu().numpy(), lam, nev)


@pytest.mark.parametrize("ozaki", [2, 1, 0])
def test_subspace_2d_each_gram_path_matches_dense(api, ozaki):
    # projection Grams on tcgen05 (2), mma.sync (1) or FP64 CUDA cores (0)
    p = pencil_2d_q1(36, seed=5)           # n = 1225
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    nev = 25
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    V0 = start_block(p.n, 38, 9)
    h = api.Handle(p, api.default_opts(gram_ozaki=ozaki))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma, torch.from_numpy(V0).cuda())
    assert st == api.OK and nconv == nev
    _check_eigs(theta.cpu().numpy(), resid.cpu().numpy(), lam, nev)
    Xh = X.cpu().numpy()[:, :nev]
    np.testing.assert_allclose(Xh.T @ (p.B() @ Xh), np.eye(nev), atol=1e-10)


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_subspace_3d_small_matches_dense(api, kernel):
    # 3-dof node groups (81 union entries each): the staged kernel's long-list
    # shape; kernel 3 takes them as 27 neighbour nodes with 3 x 3 blocks
    p = pencil_3d_elasticity(7, seed=13)   # n = 7 * 7 * 6 * 3 = 882
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    nev = 24
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    V0 = start_block(p.n, 36, 8)
    h = api.Handle(p, api.default_opts(spmm_kernel=kernel))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma, torch.from_numpy(V0).cuda())
    assert st == api.OK and nconv == nev == inertia.count_below_sparse(p.A(), p.B(), gamma)
    _check_eigs(theta.cpu().numpy(), resid.cpu().numpy(), lam, nev)


def test_subspace_host_entry_equals_device_entry(api):
    p = pencil_2d_q1(24, seed=2)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[9] + lam[10])
    f = api.Filter(*poles.quadrature_poles("gauss_legendre", 4, gamma))
    V0 = start_block(p.n, 16, 3)
    h = api.Handle(p)
    th_d, X_d, r_d, nc_d, st_d, _ = h.subspace_iterate(f, gamma, torch.from_numpy(V0).cuda())
    th_h, X_h, r_h, nc_h, st_h, _ = h.subspace_iterate_host(f, gamma, V0)
    assert st_d == st_h == api.OK and nc_d == nc_h == 10
    np.testing.assert_array_equal(th_d.cpu().numpy(), th_h)
    np.testing.assert_array_equal(X_d.cpu().numpy(), X_h)


@pytest.mark.parametrize("pinned", [False, True])
def test_subspace_host_entry_pitched_blocks(api, pinned):
    # V0 and X with row pitches above L, in pageable or pinned host memory
    # (the pageable pitched blocks go through one contiguous copy and a host
    # row gather/scatter, the pinned ones through a pitched copy): the same
    # bits as the contiguous call, and the padding columns left untouched
    import ctypes as C
    p = pencil_2d_q1(24, seed=2)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[9] + lam[10])
    f = api.Filter(*poles.quadrature_poles("gauss_legendre", 4, gamma))
    L = 16
    V0 = start_block(p.n, L, 3)
    h = api.Handle(p)
    th_c, X_c, r_c, nc_c, st_c, _ = h.subspace_iterate_host(f, gamma, V0)

    def host(shape, fill):
        if pinned:
            a = torch.full(shape, fill, dtype=torch.float64).pin_memory().numpy()
        else:
            a = np.full(shape, fill)
        return a
    ldv, ldx = L + 3, L + 5
    Vp = host((p.n, ldv), 7.0)
    Vp[:, :L] = V0
    Xp = host((p.n, ldx), -3.0)
    th, res = np.zeros(L), np.zeros(L)
    nconv = C.c_int32(0)
    rep = api.slrf_report()
    st = h.lib.slrf_subspace_iterate_host(h.h, C.byref(f.c), gamma, L, Vp.ctypes.data, ldv, 1e-8, 50,
                                          th.ctypes.data, Xp.ctypes.data, ldx, res.ctypes.data, C.byref(nconv),
                                          C.byref(rep))
    assert st == st_c == api.OK and nconv.value == nc_c
    np.testing.assert_array_equal(th, th_c)
    np.testing.assert_array_equal(Xp[:, :L], X_c)
    assert np.all(Xp[:, L:] == -3.0) and np.all(Vp[:, L:] == 7.0)


def test_release_cached_memory(api):
    # a destroyed handle's memory stays in the library's pool for the next
    # handle; the trim hands it back, and the next handle solves as before
    p = pencil_2d_q1(24, seed=2)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[9] + lam[10])
    f = api.Filter(*poles.quadrature_poles("gauss_legendre", 4, gamma))
    V0 = start_block(p.n, 16, 3)
    out = []
    for _ in range(2):
        h = api.Handle(p)
        out.append(h.subspace_iterate_host(f, gamma, V0))
        h.close()
        api.release_cached_memory(torch.cuda.current_device())
    assert out[0][4] == out[1][4] == api.OK
    np.testing.assert_array_equal(out[0][1], out[1][1])
    api.release_cached_memory(torch.cuda.device_count() + 5)   # no pool there: nothing to do


def test_subspace_too_small_is_reported(api):
    p = pencil_1d(300)
    lam = inertia.lambda_1d(300)
    gamma = lam[40]                         # 41 eigenvalues inside, subspace of 12
    f = api.Filter(*poles.quadrature_poles("midpoint", 2, gamma))
    h = api.Handle(p)
    *_, st, rep = h.subspace_iterate(f, gamma, torch.from_numpy(start_block(300, 12, 1)).cuda(), max_outer=5)
    assert st == api.SUBSPACE_TOO_SMALL


def test_stagnation_is_reported(api):
    # a single pole far outside the spectrum gives an almost constant filter:
    # the subspace stops improving, and the iteration says so instead of
    # running to max_outer
    n = 400
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[7] + lam[8])
    far = api.Filter([1e6 * gamma * (1 + 1j)], [1.0])
    V0 = torch.from_numpy(start_block(n, 12, 3)).cuda()
    h = api.Handle(p, api.default_opts(stagnation_window=4))
    *_, nconv, st, rep = h.subspace_iterate(far, gamma, V0, tol=1e-8, max_outer=40)
    assert st == api.STAGNATION
    # the mixed form first retries with FP64 Krylov solves, then gives up
    assert rep.krylov_fp64 == 1 and rep.outer_iters <= 11
    assert nconv < rep.n_wanted or rep.n_wanted == 0   # nothing converged
    h.set_opts(stagnation_window=0)
    *_, nconv, st, rep = h.subspace_iterate(far, gamma, V0, tol=1e-8, max_outer=7)
    assert st == api.NOT_CONVERGED and rep.outer_iters == 7


def test_invalid_arguments_are_rejected(api):
    p = pencil_1d(50)
    h = api.Handle(p)
    bad = api.Filter(np.array([1.0 + 0j]), np.array([1.0 + 0j]))       # pole on the real axis
    with pytest.raises(api.SlrfError):
        h.filter_apply(bad, torch.zeros((50, 2), dtype=torch.float64, device="cuda"))
    p2 = pencil_1d(50)
    p2.a_val = p2.a_val.copy()
    p2.a_val[3] = np.nan
    with pytest.raises(api.SlrfError):
        api.Handle(p2)
    p3 = pencil_1d(50)
    p3.col_idx = p3.col_idx.copy()
    p3.col_idx[[1, 2]] = p3.col_idx[[2, 1]]                              # unsorted row
    with pytest.raises(api.SlrfError):
        api.Handle(p3)


# --------------------------------------------------------------------------
# full benchmark workload (2D Q1 300 x 300, L = 150, N = 4), mixed precision
# --------------------------------------------------------------------------
def test_full_2d_config_matches_stored_oracle_spectrum(api):
    name = "fem2d_q1_300"
    p = config_pencil(name)
    iv = interval_for(name)
    lam = np.array(iv["lambda"])
    f = api.Filter(*poles.slrf_poles(4, 1.0, 0.01, iv["gamma"]))
    V0 = start_block(p.n, iv["L"], 2505)
    h = api.Handle(p)
    theta, X, resid, nconv, st, rep = h.subspace_iterate(f, iv["gamma"], torch.from_numpy(V0).cuda(),
                                                         tol=1e-8, max_outer=40)
    theta = theta.cpu().numpy()
    assert st == api.OK
    assert nconv == rep.n_wanted == iv["nev"] == iv["inertia_count"]
    _check_eigs(theta, resid.cpu().numpy(), lam, iv["nev"])
    # sampled residuals recomputed by the oracle side in FP64
    Xh = X.cpu().numpy()
    idx = np.array([0, 17, 55, 99])
    xs = Xh[:, idx]
    r = p.A() @ xs - (p.B() @ xs) * theta[idx][None, :]
    rho = np.linalg.norm(r, axis=0) / (np.abs(theta[idx]) * np.linalg.norm(p.B() @ xs, axis=0))
    assert rho.max() <= 1e-8


# --------------------------------------------------------------------------
# full 3D elasticity workload (40^3 nodes x 3 dof, one face clamped, L = 300)
# --------------------------------------------------------------------------
def test_full_3d_config_matches_stored_oracle_spectrum(api):
    name = "fem3d_elastic_40"
    p = config_pencil(name)
    iv = interval_for(name)
    lam = np.array(iv["lambda"])
    f = api.Filter(*poles.slrf_poles(4, 1.0, 0.01, iv["gamma"]))
    V0 = start_block(p.n, iv["L"], 2506)
    h = api.Handle(p)
    theta, X, resid, nconv, st, rep = h.subspace_iterate(f, iv["gamma"], torch.from_numpy(V0).cuda(),
                                                         tol=1e-8, max_outer=40)
    theta = theta.cpu().numpy()
    assert st == api.OK
    assert nconv == rep.n_wanted == iv["nev"] == iv["inertia_count"]
    _check_eigs(theta, resid.cpu().numpy(), lam, iv["nev"])
    Xh = X.cpu().numpy()
    idx = np.array([0, 1, 77, 150, 199])
    xs = Xh[:, idx]
    r = p.A() @ xs - (p.B() @ xs) * theta[idx][None, :]
    rho = np.linalg.norm(r, axis=0) / (np.abs(theta[idx]) * np.linalg.norm(p.B() @ xs, axis=0))
    assert rho.max() <= 1e-8
    np.testing.assert_allclose(xs.T @ (p.B() @ xs), np.eye(len(idx)), atol=1e-10)
