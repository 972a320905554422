"""GPU checks of the multigrid-preconditioned shifted solves (SLRF_PRECOND_MG)
through the C ABI: the preconditioner changes the Krylov iterates, never the
filter, so every variant must reproduce the oracle's filter (exact sparse LU
per pole) to the FP64 inner tolerance, and the eigenpairs of Algorithm 1."""
import numpy as np
import pytest
import scipy.linalg as la

from oracle import filter as ofilt
from oracle import poles
from workloads import pencil_1d, pencil_2d_q1, pencil_3d_elasticity, start_block

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


def _filter_case(p, nev, N=4):
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(N, 1.0, 0.01, gamma)
    return lam, gamma, s, w


@pytest.mark.parametrize("variant", [
    dict(precond=1),                                  # Jacobi
    dict(precond=2),                                  # V-cycle, default levels
    dict(precond=2, mg_coarse=16),                    # deeper hierarchy, exact solve on <= 16 unknowns
    dict(precond=2, mg_coarse=16, mg_cycle=2),        # W-cycle
    dict(precond=2, mg_coarse=16, mg_nu=1, mg_omega=1.0),
])
def test_filter_apply_fp64_each_cycle_matches_exact_lu(api, variant):
    p = pencil_2d_q1(22, seed=9)                      # n = 441
    _, _, s, w = _filter_case(p, 15)
    V = start_block(p.n, 13, 4)                       # 13 columns: odd, ragged against the 2-column groups
    h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000, **variant))
    U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), ofilt.filter_apply(p.A(), p.B(), s, w, V)) < 1e-10
    if variant["precond"] == 2:
        assert rep.as_dict()["kernels"]["mg_fine"]["launches"] > 0


def test_multigrid_cuts_the_iterations(api):
    p = pencil_2d_q1(40, seed=3)                      # n = 1521, three levels
    _, _, s, w = _filter_case(p, 20)
    V = start_block(p.n, 16, 6)
    its = {}
    for pc in (api.PRECOND_JACOBI, api.PRECOND_MG):
        h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-10, precond=pc))
        U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
        assert st == api.OK
        its[pc] = max(rep.iters_per_pole[:4])
    assert its[api.PRECOND_MG] * 3 < its[api.PRECOND_JACOBI]


def test_single_level_hierarchy_is_an_exact_solve(api):
    p = pencil_1d(200)                                # n <= 256: the coarsest level is the pencil
    assert api.mg_describe(p)["levels"] == [200]
    _, _, s, w = _filter_case(p, 8)
    V = start_block(p.n, 6, 7)
    h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-12, precond=api.PRECOND_MG))
    U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), ofilt.filter_apply(p.A(), p.B(), s, w, V)) < 1e-10
    assert max(rep.iters_per_pole[:4]) <= 3


def test_node_block_hierarchy(api):
    p = pencil_3d_elasticity(5)                       # n = 300, 3-dof nodes: row groups of 3 on the finest level
    _, _, s, w = _filter_case(p, 10)
    V = start_block(p.n, 8, 8)
    # 1e-13 like the other FP64 filter checks: this pencil's shifted systems are
    # worse conditioned, so 1e-12 leaves ~1.2e-10 in the solution (Jacobi too)
    o = api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000, precond=api.PRECOND_MG,
                         mg_coarse=30)
    assert len(api.mg_describe(p, o)["levels"]) >= 2
    h = api.Handle(p, o)
    U, st, _ = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), ofilt.filter_apply(p.A(), p.B(), s, w, V)) < 1e-10


def test_switching_to_multigrid_builds_the_hierarchy_lazily(api):
    p = pencil_2d_q1(22, seed=9)
    _, _, s, w = _filter_case(p, 15)
    V = torch.from_numpy(start_block(p.n, 10, 4)).cuda()
    h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, precond=api.PRECOND_JACOBI))
    U1, st1, _ = h.filter_apply(api.Filter(s, w), V)
    h.set_opts(precond=api.PRECOND_MG)
    U2, st2, rep = h.filter_apply(api.Filter(s, w), V)
    assert st1 == st2 == api.OK
    assert "mg_fine" in rep.as_dict()["kernels"]
    assert rel_err(U2.cpu().numpy(), U1.cpu().numpy()) < 1e-10


def test_hierarchy_built_behind_handle_creation(api):
    # slrf_create returns before the host hierarchy is ready: a handle
    # destroyed at once waits for its setup thread; one whose options change
    # before the first solve finishes the pending build first, then rebuilds
    # with the new coarsening; results equal a handle that had it ready
    p = pencil_2d_q1(60, seed=4)
    for _ in range(3):
        api.Handle(p, api.default_opts(precond=api.PRECOND_MG)).close()
    _, _, s, w = _filter_case(p, 15)
    V = torch.from_numpy(start_block(p.n, 8, 2)).cuda()
    o = dict(precision=api.PREC_FP64, inner_tol=1e-13, precond=api.PRECOND_MG)
    h1 = api.Handle(p, api.default_opts(**o))
    h1.set_opts(mg_coarse=64)
    U1, st1, rep1 = h1.filter_apply(api.Filter(s, w), V)
    h2 = api.Handle(p, api.default_opts(mg_coarse=64, **o))
    U2, st2, rep2 = h2.filter_apply(api.Filter(s, w), V)
    assert st1 == st2 == api.OK and rep1.mg_levels == rep2.mg_levels
    np.testing.assert_array_equal(U1.cpu().numpy(), U2.cpu().numpy())


@pytest.mark.parametrize("precond", ["JACOBI", "MG"])
def test_subspace_2d_each_preconditioner_matches_dense(api, precond):
    p = pencil_2d_q1(40, seed=5)
    lam, gamma, s, w = _filter_case(p, 25)
    h = api.Handle(p, api.default_opts(precond=getattr(api, "PRECOND_" + precond)))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma,
                                                         torch.from_numpy(start_block(p.n, 38, 11)).cuda(),
                                                         tol=1e-8, max_outer=30)
    assert st == api.OK and nconv == rep.n_wanted == 25
    th = theta.cpu().numpy()[:25]
    assert np.max(np.abs(th - lam[:25]) / lam[:25]) < 1e-10


def test_deep_shift_truncates_the_cycle(api):
    # |sigma| max(b_ii/a_ii) passes 0.8 on level 1 (725 unknowns): the cycle
    # stops there and solves that level exactly
    p = pencil_2d_q1(80, seed=7)                      # levels 6241, 725, 107
    s, w = poles.slrf_poles(4, 1.0, 0.01, 3500.0)
    V = start_block(p.n, 6, 3)
    ref = ofilt.filter_apply(p.A(), p.B(), s, w, V)
    levels = {}
    for limit in (0.8, 100.0):
        h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000,
                                           precond=api.PRECOND_MG, mg_shift_limit=limit))
        U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
        assert st == api.OK
        assert rel_err(U.cpu().numpy(), ref) < 1e-10
        levels[limit] = rep.mg_levels
    assert levels[0.8] == 2 and levels[100.0] == 3


def test_auto_uses_jacobi_when_the_exact_level_is_too_large(api):
    p = pencil_2d_q1(120, seed=7)                     # levels 14161, 1610, 226
    s, w = poles.slrf_poles(4, 1.0, 0.01, 8000.0)     # level 1 (1610 > 768) would need the exact solve
    V = torch.from_numpy(start_block(p.n, 4, 3)).cuda()
    got = {}
    for pc in (api.PRECOND_AUTO, api.PRECOND_MG):
        h = api.Handle(p, api.default_opts(precond=pc, inner_maxit=3000))
        U, st, rep = h.filter_apply(api.Filter(s, w), V, allowed=(api.OK, api.NOT_CONVERGED))
        got[pc] = (st, rep.mg_levels)
    # AUTO solves with Jacobi; forcing the full cycle smooths the shifted
    # operator where it no longer can, and its deepest pole misses the cap
    assert got[api.PRECOND_AUTO] == (api.OK, 0)
    assert got[api.PRECOND_MG][1] == 3


def test_unattainable_tolerance_ends_in_stagnation_after_fp64(api):
    # 1D, n = 20 000: the eigenvector of lambda_1 cannot be stored in FP64 with
    # a residual below ~eps lambda_max / lambda_1 = 5e-8, so rho <= 1e-8 is out
    # of reach for it.  The mixed iteration retries with FP64 Krylov solves,
    # then reports stagnation with the pairs it did converge.
    from oracle import inertia
    n = 20000
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n, np.arange(1, 13))
    gamma = 0.5 * (lam[9] + lam[10])
    f = api.Filter(*poles.slrf_poles(4, 1.0, 0.01, gamma))
    h = api.Handle(p)
    theta, X, resid, nconv, st, rep = h.subspace_iterate(f, gamma, torch.from_numpy(start_block(n, 16, 4)).cuda(),
                                                         tol=1e-8, max_outer=60)
    assert st == api.STAGNATION and rep.krylov_fp64 == 1
    r = resid.cpu().numpy()[:10]
    assert nconv == int(np.sum(r <= 1e-8)) and 3 <= nconv < 10
    floor = 2.2e-16 * lam_max_1d(n) / lam[0]
    assert r[0] < 20 * floor
    th = theta.cpu().numpy()[:10]
    # Ritz values of pairs with residual rho are within ~rho of the eigenvalues
    assert np.max(np.abs(th - lam[:10]) / lam[:10]) < 5e-7


def lam_max_1d(n):
    from oracle import inertia
    return float(inertia.lambda_1d(n, np.array([n]))[0])


# ---------------------------------------------------------------------------
# one cycle, compared with a plain scipy model of it
# ---------------------------------------------------------------------------
def _hierarchy_model(api, p, o):
    """Level pencils (A_l, B_l) chained by Galerkin products of the library's
    prolongators, and the rho_l of its Jacobi damping."""
    import scipy.sparse as sp
    As, Bs, Ps, rhos = [p.A().tocsr()], [p.B().tocsr()], [], []
    for l in range(len(api.mg_describe(p, o)["levels"]) - 1):
        (ptr, col, val, nr, nc), rho = api.mg_transfer(p, l, o)
        P = sp.csr_matrix((val, col, ptr), shape=(nr, nc))
        Ps.append(P)
        rhos.append(rho)
        As.append((P.T @ As[-1] @ P).tocsr())
        Bs.append((P.T @ Bs[-1] @ P).tocsr())
    return As, Bs, Ps, rhos


def _cycle_model(H, o, sig, r, l, c, nu=None):
    """The cycle as written in the textbook: damped Jacobi D = (omega/rho_l) /
    diag(A_l - sigma B_l), nu sweeps per side below the finest level (one
    there), gamma coarse visits, exact solve on level c.  nu: o.mg_nu, whose
    0 (auto) means two unless the caller says otherwise (one when an FP32
    cycle ends at its dense-inverse level)."""
    if nu is None:
        nu = o.mg_nu if o.mg_nu > 0 else 2
    As, Bs, Ps, rhos = H
    M = (As[l] - sig * Bs[l]).tocsr()
    if l == c:
        return np.linalg.solve(M.toarray(), r)
    D = (o.mg_omega / rhos[l]) / (As[l].diagonal() - sig * Bs[l].diagonal())
    P = Ps[l]
    if l == 0:
        x = D * r
        e = _cycle_model(H, o, sig, P.T @ (r - M @ x), 1, c, nu)
        z1 = x + P @ e
        return z1 + D * (r - M @ z1)
    z = D * r
    for _ in range(nu - 1):
        z = z + D * (r - M @ z)
    for _ in range(o.mg_cycle):
        z = z + P @ _cycle_model(H, o, sig, P.T @ (r - M @ z), l + 1, c, nu)
    for _ in range(nu):
        z = z + D * (r - M @ z)
    return z


def _apply_case(api, p, o, s, w, prec, m=3, ldp=4, seed=0):
    N = len(s)
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((p.n, N * ldp)) + 1j * rng.standard_normal((p.n, N * ldp))
    dt = torch.complex128 if prec == api.PREC_FP64 else torch.complex64
    Rd = torch.from_numpy(R).to(dt).cuda()
    mu = torch.zeros(N * m, dtype=dt, device="cuda")
    h = api.Handle(p, o)
    Z, lv = h.precond_apply(api.Filter(s, w), Rd, m, ldp, prec=prec, mu=mu)
    R = Rd.cpu().numpy().astype(np.complex128)     # the model starts from the same (rounded) input
    return R, Z.cpu().numpy().astype(np.complex128), mu.cpu().numpy().astype(np.complex128), lv


@pytest.mark.parametrize("variant", [
    dict(),                                           # two levels (441, 57): exact solve on 57
    dict(mg_coarse=16),                               # three levels, V-cycle
    dict(mg_coarse=16, mg_cycle=2),                   # W-cycle
    dict(mg_coarse=16, mg_nu=1, mg_omega=1.0),
    dict(mg_coarse=16, mg_nu=3, mg_shift_limit=100.0),
])
def test_precond_apply_fp64_is_the_cycle(api, variant):
    p = pencil_2d_q1(22, seed=9)
    _, _, s, w = _filter_case(p, 15)
    o = api.default_opts(precision=api.PREC_FP64, precond=api.PRECOND_MG, **variant)
    H = _hierarchy_model(api, p, o)
    m, ldp = 3, 4
    R, Z, mu, lv = _apply_case(api, p, o, s, w, api.PREC_FP64, m, ldp)
    assert 2 <= lv <= len(H[0])
    for j, sig in enumerate(s):
        for c in range(m):
            col = j * ldp + c
            ref = _cycle_model(H, o, sig, R[:, col], 0, lv - 1)
            assert np.linalg.norm(Z[:, col] - ref) <= 1e-12 * np.linalg.norm(ref)
            assert abs(mu[j * m + c] - R[:, col] @ ref) <= 1e-12 * np.linalg.norm(R[:, col]) * np.linalg.norm(ref)


def test_precond_apply_mixed_is_the_cycle_in_fp32(api):
    p = pencil_2d_q1(40, seed=5)                      # n = 1521, three levels
    _, _, s, w = _filter_case(p, 25)
    o = api.default_opts(precond=api.PRECOND_MG, mg_coarse=64)
    H = _hierarchy_model(api, p, o)
    R, Z, mu, lv = _apply_case(api, p, o, s, w, api.PREC_MIXED, m=5, ldp=6, seed=2)
    assert 2 <= lv <= len(H[0])
    for j, sig in enumerate(s):
        for c in range(5):
            col = j * 6 + c
            ref = _cycle_model(H, o, sig, R[:, col], 0, lv - 1)
            assert np.linalg.norm(Z[:, col] - ref) <= 2e-5 * np.linalg.norm(ref)


def test_precond_apply_is_complex_symmetric(api):
    # x^T C y = y^T C x (unconjugated), the property COCG needs of C
    p = pencil_2d_q1(30, seed=4)
    _, _, s, w = _filter_case(p, 20)
    o = api.default_opts(precision=api.PREC_FP64, precond=api.PRECOND_MG, mg_coarse=16, mg_cycle=2)
    R, Z, _, _ = _apply_case(api, p, o, s, w, api.PREC_FP64, m=2, ldp=2, seed=3)
    for j in range(len(s)):
        x, y = R[:, 2 * j], R[:, 2 * j + 1]
        Cx, Cy = Z[:, 2 * j], Z[:, 2 * j + 1]
        assert abs(x @ Cy - y @ Cx) <= 1e-12 * abs(x @ Cy)


def test_precond_apply_truncated_cycle(api):
    # deep shift: the cycle stops at level 1 (725 unknowns) and solves it exactly
    p = pencil_2d_q1(80, seed=7)
    s, w = poles.slrf_poles(4, 1.0, 0.01, 3500.0)
    o = api.default_opts(precision=api.PREC_FP64, precond=api.PRECOND_MG)
    H = _hierarchy_model(api, p, o)
    R, Z, _, lv = _apply_case(api, p, o, s, w, api.PREC_FP64, m=2, ldp=2, seed=5)
    assert lv == 2
    for j, sig in enumerate(s):
        ref = _cycle_model(H, o, sig, R[:, 2 * j + 1], 0, 1)
        assert np.linalg.norm(Z[:, 2 * j + 1] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_precond_apply_single_level_and_jacobi(api):
    p = pencil_1d(200)                                # one level: the exact shifted solve
    _, _, s, w = _filter_case(p, 8)
    A, B = p.A().tocsr(), p.B().tocsr()
    for pc in (api.PRECOND_MG, api.PRECOND_JACOBI, api.PRECOND_NONE):
        o = api.default_opts(precision=api.PREC_FP64, precond=pc)
        R, Z, mu, lv = _apply_case(api, p, o, s, w, api.PREC_FP64, m=2, ldp=2, seed=6)
        assert lv == (1 if pc == api.PRECOND_MG else 0)
        for j, sig in enumerate(s):
            r = R[:, 2 * j]
            if pc == api.PRECOND_MG:
                ref = np.linalg.solve((A - sig * B).toarray(), r)
            elif pc == api.PRECOND_JACOBI:
                ref = r / (A.diagonal() - sig * B.diagonal())
            else:
                ref = r
            assert np.linalg.norm(Z[:, 2 * j] - ref) <= 1e-12 * np.linalg.norm(ref)
            assert abs(mu[2 * j] - r @ ref) <= 1e-12 * np.linalg.norm(r) * np.linalg.norm(ref)


def test_profile_mask_times_only_the_selected_classes(api):
    p = pencil_2d_q1(40, seed=5)
    _, _, s, w = _filter_case(p, 20)
    V = torch.from_numpy(start_block(p.n, 12, 2)).cuda()
    names = [api.class_name(i) for i in range(api.NKERNEL_CLASSES)]
    sel = {"mg_fine", "shifted_spmm"}
    mask = sum(1 << i for i, nm in enumerate(names) if nm in sel)
    h = api.Handle(p, api.default_opts(profile=1, profile_mask=mask))
    _, st, rep = h.filter_apply(api.Filter(s, w), V)
    assert st == api.OK
    k = rep.as_dict()["kernels"]
    assert all(v["ms"] > 0 for nm, v in k.items() if nm in sel)
    assert all(v["ms"] == 0 for nm, v in k.items() if nm not in sel)
    assert {"krylov_update", "mg_coarse"} <= set(k)           # launches are counted either way
    h.set_opts(profile_mask=0)                                # 0: every class
    _, _, rep = h.filter_apply(api.Filter(s, w), V)
    assert all(v["ms"] > 0 for v in rep.as_dict()["kernels"].values())


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("mg_exact,level,m,ldp", [(1536, 2, 3, 4), (2000, 1, 3, 4), (1536, 2, 70, 70),
                                                  (1536, 2, 150, 150)])
def test_precond_apply_mixed_exact_inverse_level(api, mg_exact, level, m, ldp, tc):
    # FP32 cycle ending at a level solved by its dense shifted inverses,
    # formed on the GPU by blocked Gauss-Jordan: levels 16641 -> 1899 -> 260 -> 41;
    # the inverses applied on the tensor cores (tc = 1: three-way bf16 split,
    # one N tile of 16 / 80 / 160 columns) or by cuBLAS (tc = 0)
    from workloads import weyl_gamma
    p = pencil_2d_q1(130, seed=5)
    # poles for an interval of ~40 eigenvalues (the apply needs no exact gap)
    s, w = poles.slrf_poles(4, 1.0, 0.01, weyl_gamma("2d", 40))
    o = api.default_opts(precond=api.PRECOND_MG, mg_exact=mg_exact, mg_exact_tc=tc)
    H = _hierarchy_model(api, p, o)
    assert [A.shape[0] for A in H[0]] == [16641, 1899, 260, 41]
    R, Z, mu, lv = _apply_case(api, p, o, s, w, api.PREC_MIXED, m=m, ldp=ldp, seed=6)
    assert lv == level + 1
    for j, sig in enumerate(s):
        for c in sorted({0, 1, m // 2, m - 1}):
            col = j * ldp + c
            ref = _cycle_model(H, o, sig, R[:, col], 0, level, nu=o.mg_nu or 1)
            assert np.linalg.norm(Z[:, col] - ref) <= 5e-4 * np.linalg.norm(ref)
    # complex symmetric up to FP32 rounding: x^T C y = y^T C x
    for j in range(len(s)):
        x, y = R[:, ldp * j], R[:, ldp * j + 1]
        Cx, Cy = Z[:, ldp * j], Z[:, ldp * j + 1]
        assert abs(x @ Cy - y @ Cx) <= 1e-4 * abs(x @ Cy)


@pytest.mark.parametrize("mg_exact,tc", [(1536, 1), (1536, 0), (0, 1)])
def test_subspace_2d_with_and_without_the_exact_inverse_level(api, mg_exact, tc):
    p = pencil_2d_q1(60, seed=12)                     # levels 3481 -> 402 -> 66
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    nev = 30
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    V0 = start_block(p.n, 45, 13)
    h = api.Handle(p, api.default_opts(precond=api.PRECOND_MG, mg_exact=mg_exact, mg_exact_tc=tc))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma, torch.from_numpy(V0).cuda())
    assert st == api.OK and nconv == nev
    assert rep.mg_levels == (2 if mg_exact else 3)
    th = theta.cpu().numpy()[:nev]
    assert np.max(np.abs(th - lam[:nev]) / lam[:nev]) <= 1e-10
    assert resid.cpu().numpy()[:nev].max() <= 1e-8
