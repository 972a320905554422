"""GPU checks of the BiCGStab variant of the shifted solves (SLRF_KRYLOV_BICGSTAB,
the paper's Krylov method, Section 4.2.1) through the C ABI: with either
preconditioner it must reproduce the oracle's filter (exact sparse LU per
pole) to the FP64 inner tolerance, and Algorithm 1's eigenpairs."""
import numpy as np
import pytest
import scipy.linalg as la

from oracle import filter as ofilt
from oracle import poles
from workloads import pencil_1d, pencil_2d_q1, start_block

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


def _case(p, nev, N=4):
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    s, w = poles.slrf_poles(N, 1.0, 0.01, gamma)
    return lam, gamma, s, w


@pytest.mark.parametrize("precond", ["JACOBI", "MG"])
def test_bicgstab_filter_fp64_matches_exact_lu(api, precond):
    p = pencil_2d_q1(22, seed=9)                      # n = 441
    _, _, s, w = _case(p, 15)
    V = start_block(p.n, 13, 4)
    o = api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000, krylov=api.KRYLOV_BICGSTAB,
                         precond=getattr(api, "PRECOND_" + precond))
    h = api.Handle(p, o)
    U, st, rep = h.filter_apply(api.Filter(s, w), torch.from_numpy(V).cuda())
    assert st == api.OK
    assert rel_err(U.cpu().numpy(), ofilt.filter_apply(p.A(), p.B(), s, w, V)) < 1e-10
    # two shifted products per BiCGStab iteration
    its = sum(rep.iters_per_pole[:4]) * V.shape[1]
    assert rep.spmv == pytest.approx(2 * its, rel=1e-9)


def test_bicgstab_equals_cocg_filter(api):
    p = pencil_1d(400)
    _, _, s, w = _case(p, 10)
    V = torch.from_numpy(start_block(p.n, 8, 2)).cuda()
    out = {}
    for kr in (api.KRYLOV_COCG, api.KRYLOV_BICGSTAB):
        h = api.Handle(p, api.default_opts(precision=api.PREC_FP64, inner_tol=1e-13, inner_maxit=3000, krylov=kr))
        U, st, _ = h.filter_apply(api.Filter(s, w), V)
        assert st == api.OK
        out[kr] = U.cpu().numpy()
    assert rel_err(out[api.KRYLOV_BICGSTAB], out[api.KRYLOV_COCG]) < 1e-10


@pytest.mark.parametrize("precond", ["JACOBI", "MG"])
def test_bicgstab_subspace_mixed_matches_dense(api, precond):
    p = pencil_2d_q1(40, seed=5)
    lam, gamma, s, w = _case(p, 25)
    h = api.Handle(p, api.default_opts(krylov=api.KRYLOV_BICGSTAB, precond=getattr(api, "PRECOND_" + precond)))
    theta, X, resid, nconv, st, rep = h.subspace_iterate(api.Filter(s, w), gamma,
                                                         torch.from_numpy(start_block(p.n, 38, 11)).cuda(),
                                                         tol=1e-8, max_outer=30)
    assert st == api.OK and nconv == rep.n_wanted == 25
    th = theta.cpu().numpy()[:25]
    assert np.max(np.abs(th - lam[:25]) / lam[:25]) < 1e-10
