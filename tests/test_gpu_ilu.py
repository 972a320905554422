"""The ILU preconditioner (SLRF_PRECOND_ILU): the paper's Krylov
preconditioner (Section 4.2.1) in a no-fill, fixed-point form, through the
C ABI.  One application is checked against a plain scipy model of the same
operator (fixed-point factor sweeps, Jacobi sweeps of the triangular
solves); whole filters against the oracle's exact sparse LU."""
import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp

from oracle import filter as ofilt
from oracle import inertia, poles
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


def _poles_for(p, nev, N=4):
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(N, 1.0, 0.01, gamma)
    return lam, gamma, s, w


def _ilu_model(p, sig, sweeps):
    """No-fill L D L^T of M = A - sig B on the pencil's pattern by fixed-point
    sweeps: l_ik = (m_ik - (L D L^T)_ik) / d_k, d_i = m_ii - (L D L^T)_ii with
    the right-hand sides from the previous iterate (L strictly lower here)."""
    M = sp.csr_matrix((p.a_val - sig * p.b_val, p.col_idx, p.row_ptr), shape=(p.n, p.n))
    M.sort_indices()
    mask = sp.tril(M, k=-1).tocsr()
    mask.data[:] = 1.0
    dM = M.diagonal()
    L = sp.tril(M, k=-1).tocsr().multiply(1.0 / dM[None, :]).tocsr()
    D = dM.copy()
    for _ in range(sweeps):
        S = (L @ sp.diags(D) @ L.T).tocsr()
        Ln = (sp.tril(M, k=-1) - S.multiply(mask)).tocsr().multiply(1.0 / D[None, :]).tocsr()
        Dn = dM - S.diagonal()
        L, D = Ln, Dn
    return L.tocsr(), D


def _ilu_apply_model(L, D, r, tri):
    y = r.copy()
    for _ in range(tri):
        y = r - L @ y
    w = y / D
    z = w.copy()
    for _ in range(tri):
        z = w - L.T @ z
    return z


def _apply(api, p, o, s, w, m=3, ldp=4, seed=0):
    N = len(s)
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((p.n, N * ldp)) + 1j * rng.standard_normal((p.n, N * ldp))
    Rd = torch.from_numpy(R).to(torch.complex128).cuda()
    mu = torch.zeros(N * m, dtype=torch.complex128, device="cuda")
    h = api.Handle(p, o)
    Z, lv = h.precond_apply(api.Filter(s, w), Rd, m, ldp, prec=api.PREC_FP64, mu=mu)
    return R, Z.cpu().numpy(), mu.cpu().numpy(), lv


@pytest.mark.parametrize("sweeps,tri", [(0, 1), (3, 3), (2, 4)])
@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_precond_apply_ilu_is_the_model(api, kind, sweeps, tri):
    p = pencil_2d_q1(20, seed=3) if kind == "2d" else pencil_3d_elasticity(5, seed=4)
    _, _, s, w = _poles_for(p, 12)
    o = api.default_opts(precision=api.PREC_FP64, precond=api.PRECOND_ILU, ilu_sweeps=sweeps, ilu_tri_sweeps=tri)
    R, Z, mu, lv = _apply(api, p, o, s, w)
    assert lv == 0
    for j, sig in enumerate(s):
        L, D = _ilu_model(p, sig, sweeps)
        for c in range(3):
            col = j * 4 + c
            ref = _ilu_apply_model(L, D, R[:, col], tri)
            assert rel_err(Z[:, col], ref) <= 1e-12
            assert abs(mu[j * 3 + c] - R[:, col] @ ref) <= 1e-12 * np.linalg.norm(R[:, col]) * np.linalg.norm(ref)


def test_precond_apply_ilu_is_complex_symmetric(api):
    # x^T C y = y^T C x (unconjugated), what COCG needs of its preconditioner
    p = pencil_2d_q1(26, seed=8)
    _, _, s, w = _poles_for(p, 20)
    o = api.default_opts(precision=api.PREC_FP64, precond=api.PRECOND_ILU)
    R, Z, _, _ = _apply(api, p, o, s, w, m=2, ldp=2, seed=3)
    for j in range(len(s)):
        x, y = R[:, 2 * j], R[:, 2 * j + 1]
        Cx, Cy = Z[:, 2 * j], Z[:, 2 * j + 1]
        assert abs(x @ Cy - y @ Cx) <= 1e-12 * abs(x @ Cy)


@pytest.mark.parametrize("krylov", ["COCG", "BICGSTAB"])
@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_filter_apply_fp64_ilu_matches_exact_lu(api, krylov, kind):
    p = pencil_2d_q1(22, seed=9) if kind == "2d" else pencil_3d_elasticity(6, seed=5)
    _, _, s, w = _poles_for(p, 15)
    V = start_block(p.n, 13, 4)
    o = api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000, precond=api.PRECOND_ILU,
                         krylov=getattr(api, "KRYLOV_" + krylov))
    h = api.Handle(p, o)
    U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), ofilt.filter_apply(p.A(), p.B(), s, w, V)) < 1e-10


def test_ilu_cuts_the_iterations_against_jacobi(api):
    p = pencil_2d_q1(40, seed=3)                      # n = 1521
    _, _, s, w = _poles_for(p, 20)
    V = start_block(p.n, 16, 6)
    its = {}
    for pc in (api.PRECOND_JACOBI, api.PRECOND_ILU):
        h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-10, precond=pc))
        U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
        assert st == api.OK
        its[pc] = max(rep.iters_per_pole[:4])
    assert its[api.PRECOND_ILU] < its[api.PRECOND_JACOBI]


@pytest.mark.parametrize("krylov", ["COCG", "BICGSTAB"])
def test_subspace_mixed_with_ilu_matches_the_closed_form(api, krylov):
    n = 600
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[11] + lam[12])
    s, w = poles.slrf_poles(2, 1.0, 0.01, gamma)
    V0 = torch.from_numpy(start_block(n, 18, 5)).cuda()
    h = api.Handle(p, api.default_opts(precond=api.PRECOND_ILU, krylov=getattr(api, "KRYLOV_" + krylov)))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma, V0, tol=1e-8, max_outer=30)
    assert st == api.OK and nconv == 12 == inertia.count_below_1d(n, gamma)
    th = theta.cpu().numpy()[:12]
    assert np.max(np.abs(th - lam[:12]) / lam[:12]) <= 1e-10
    assert resid.cpu().numpy()[:12].max() <= 1e-8
