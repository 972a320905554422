"""Pins for the FP64 oracle: closed forms, brute force, identities, paper facts.

Each test ties the oracle to something other than itself, so that a dropped
term, a wrong sign or index, or a transposed operand in it fails here.
"""
import numpy as np
import pytest
import scipy.linalg as la

from oracle import filter as ofilt
from oracle import inertia, poles, rr, subspace
from workloads import pencil_1d, pencil_2d_q1, pencil_3d_elasticity, start_block


# --------------------------------------------------------------------------
# closed-form spectra (Section 1 notation; 1D/2D uniform FEM)
# --------------------------------------------------------------------------
def test_lambda_1d_closed_form_matches_dense():
    p = pencil_1d(60)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    np.testing.assert_allclose(lam, inertia.lambda_1d(60), rtol=1e-11)


def test_lambda_1d_printed_values():
    # lambda_1, lambda_20 and lambda_21 at n = 2000 (h = 1/2001), as evaluated
    # from the closed form (6/h^2)(1-cos k pi h)/(2+cos k pi h).
    lam = inertia.lambda_1d(2000, [1, 20, 21])
    np.testing.assert_allclose(lam, [9.869606428, 3948.166144, 4352.889832], rtol=1e-9)
    # lambda_1 tends to pi^2 as h -> 0 (continuous Dirichlet Laplacian).
    assert abs(lam[0] - np.pi ** 2) / np.pi ** 2 < 1e-5


def test_lambda_2d_unit_tensor_sum_matches_dense():
    m = 10
    p = pencil_2d_q1(m, seed=None)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    np.testing.assert_allclose(lam, inertia.lambda_2d_unit(m), rtol=1e-10)


def test_eigvec_1d_is_eigenvector():
    n, k = 50, 7
    p = pencil_1d(n)
    x = inertia.eigvec_1d(n, k)
    r = p.A() @ x - inertia.lambda_1d(n, k) * (p.B() @ x)
    assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(p.A() @ x)


# --------------------------------------------------------------------------
# Sylvester inertia counts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("gamma_index", [1, 5, 20, 37])
def test_sturm_count_1d(gamma_index):
    n = 80
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[gamma_index - 1] + lam[gamma_index])
    assert inertia.count_below_1d(n, gamma) == gamma_index
    p = pencil_1d(n)
    assert inertia.count_below_dense(p.A(), p.B(), gamma) == gamma_index
    assert inertia.count_below_sparse(p.A(), p.B(), gamma) == gamma_index


def test_sparse_and_dense_counts_2d_lognormal():
    p = pencil_2d_q1(14, seed=11)
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    for k in (3, 17, 60):
        gamma = 0.5 * (lam[k - 1] + lam[k])
        assert inertia.count_below_dense(p.A(), p.B(), gamma) == k
        assert inertia.count_below_sparse(p.A(), p.B(), gamma) == k


# --------------------------------------------------------------------------
# rational filters (Section 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 4, 8])
def test_midpoint_filter_closed_form(N):
    # 2N nodes at the roots of z^{2N} = -1 on the circle (c, r): the midpoint
    # rule gives exactly Phi(x) = 1 / (1 + ((x - c)/r)^{2N}).
    gamma = 3.7
    s, w = poles.quadrature_poles("midpoint", N, gamma)
    x = np.linspace(-2.0, 3 * gamma, 301)
    c = r = gamma / 2
    np.testing.assert_allclose(poles.phi_real(x, s, w), 1.0 / (1.0 + ((x - c) / r) ** (2 * N)),
                               rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_gauss_legendre_centre_and_endpoint(N):
    gamma = 2.0
    s, w = poles.quadrature_poles("gauss_legendre", N, gamma)
    # centre: the rule integrates the resolvent of the centre exactly (=1);
    # the endpoints lie on the contour, where the two halves contribute 1/2.
    assert abs(poles.phi_real([gamma / 2], s, w)[0] - 1.0) < 1e-13
    assert abs(poles.phi_real([gamma], s, w)[0] - 0.5) < 1e-13
    assert abs(poles.phi_real([0.0], s, w)[0] - 0.5) < 1e-13


def test_quadrature_pole_geometry_n3():
    # Section 3.2 / Table 4: the middle pole is shared by the three rules, and
    # the Gauss-Chebyshev outer poles are closest to the real axis.
    sm, _ = poles.quadrature_poles("midpoint", 3, 1.0)
    sl, _ = poles.quadrature_poles("gauss_legendre", 3, 1.0)
    sc, _ = poles.quadrature_poles("gauss_chebyshev", 3, 1.0)
    np.testing.assert_allclose([sm[1], sl[1], sc[1]], [0.5 + 0.5j] * 3, atol=1e-14)
    assert sc[2].imag < sl[2].imag < sm[2].imag
    # separation factors: Gauss-Chebyshev steepest (Section 3.2).
    f = [poles.separation_factor(*poles.quadrature_poles(r, 3, 1.0), 1.0)
         for r in ("midpoint", "gauss_legendre", "gauss_chebyshev")]
    assert f[0] < f[1] < f[2]
    np.testing.assert_allclose(f[0], 3.0, rtol=1e-12)   # d/dx of 1/(1+t^6) at t=1 is -6/4 /r


def test_slrf_design_properties():
    gamma = 5.0
    s, w = poles.slrf_poles(4, 1.0, 0.01, gamma)
    # poles on the line x (1 + i alpha) with x in (0, gamma]
    np.testing.assert_allclose(s.imag, s.real * 1.0, rtol=1e-12)
    assert np.all(s.real > 0) and np.all(s.real <= gamma)
    # conjugate symmetry Phi(conj z) = conj Phi(z); real on the real axis
    z = np.array([0.3 + 0.7j, 4.0 - 1.0j, 9.0 + 0.1j])
    np.testing.assert_allclose(poles.phi(np.conj(z), s, w), np.conj(poles.phi(z, s, w)), rtol=1e-13)
    assert np.max(np.abs(poles.phi(np.array([1.0, 6.0]), s, w).imag)) < 1e-14
    # scaling: Phi_gamma(x) = Phi_1(x / gamma)
    s1, w1 = poles.slrf_poles(4, 1.0, 0.01, 1.0)
    x = np.linspace(0, 3 * gamma, 50)
    np.testing.assert_allclose(poles.phi_real(x, s, w), poles.phi_real(x / gamma, s1, w1),
                               rtol=1e-9, atol=1e-12)
    # passes the wanted interval, damps the far tail (Section 3.1 objective)
    assert poles.phi_real([0.5], s1, w1)[0] > 0.8
    assert abs(poles.phi_real([3.0], s1, w1)[0]) < 0.05


def test_slrf_separation_grows_with_n_and_falls_with_alpha():
    # Figure 2/3 text: |Phi'(gamma)| increases with N and decreases with alpha.
    seps = [poles.separation_factor(*poles.slrf_poles(N, 1.0, 0.01), 1.0) for N in (1, 2, 4, 8)]
    assert all(a < b for a, b in zip(seps, seps[1:]))
    sa = [poles.separation_factor(*poles.slrf_poles(4, a, 1.0), 1.0) for a in (0.5, 1.0, 2.0)]
    assert sa[0] > sa[1] > sa[2]


def test_prop21_condition_number_closed_form():
    # Proposition 2.1: kappa(B^{-1}(A - sigma B)) from the extreme eigenvalues.
    p = pencil_1d(40)
    lam = inertia.lambda_1d(40)
    mu = 0.5 * (lam[3] + lam[4]) + 0.3 * (lam[4] - lam[3])
    prev = np.inf
    for alpha in (0.05, 0.5, 1.0):
        sigma = mu * (1 + 1j * alpha)
        ev = la.eigvals(la.solve(p.B().toarray(), p.A().toarray() - sigma * p.B().toarray()))
        kappa = np.abs(ev).max() / np.abs(ev).min()
        far = lam[np.argmax(np.abs(lam - mu))]
        near = lam[np.argmin(np.abs(lam - mu))]
        closed = np.sqrt((far - mu) ** 2 + (alpha * mu) ** 2) / np.sqrt((near - mu) ** 2 + (alpha * mu) ** 2)
        np.testing.assert_allclose(kappa, closed, rtol=1e-8)
        assert closed < prev
        prev = closed


# --------------------------------------------------------------------------
# filter operator with exact solves (Section 3, Algorithm 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rule", ["slrf", "midpoint", "gauss_legendre"])
def test_filter_acts_on_eigenvectors_by_phi(rule):
    # Phi(A, B) x_i = Phi(lambda_i) x_i (Section 3, eigen-decomposition of v).
    n = 300
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[9] + lam[10])
    if rule == "slrf":
        s, w = poles.slrf_poles(3, 1.0, 0.01, gamma)
    else:
        s, w = poles.quadrature_poles(rule, 4, gamma)
    ks = [1, 4, 10, 11, 15, 40]
    V = np.stack([inertia.eigvec_1d(n, k) for k in ks], axis=1)
    U = ofilt.filter_apply(p.A(), p.B(), s, w, V)
    expect = V * poles.phi_real(lam[np.array(ks) - 1], s, w)[None, :]
    np.testing.assert_allclose(U, expect, rtol=0, atol=1e-11 * np.abs(V).max())


def test_corrected_form_equals_plain_form():
    # The residual-corrected identity holds for any X and real Theta.
    n = 400
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[11] + lam[12])
    s, w = poles.slrf_poles(2, 1.0, 0.01, gamma)
    X = start_block(n, 9, 5)
    theta = np.linspace(0.1, 2.0, 9) * gamma
    U1 = ofilt.filter_apply(p.A(), p.B(), s, w, X)
    U2 = ofilt.filter_apply_corrected(p.A(), p.B(), s, w, X, theta)
    assert np.linalg.norm(U1 - U2) < 1e-12 * np.linalg.norm(U1)


def test_filter_is_linear_and_real():
    p = pencil_2d_q1(9, seed=3)
    s, w = poles.quadrature_poles("gauss_legendre", 3, 500.0)
    V = start_block(p.n, 4, 9)
    U = ofilt.filter_apply(p.A(), p.B(), s, w, V)
    U2 = ofilt.filter_apply(p.A(), p.B(), s, w, 2.0 * V[:, ::-1])
    np.testing.assert_allclose(U2, 2.0 * U[:, ::-1], rtol=1e-12, atol=1e-14)
    assert U.dtype == np.float64


# --------------------------------------------------------------------------
# Rayleigh-Ritz and Algorithm 1
# --------------------------------------------------------------------------
def test_rayleigh_ritz_on_exact_subspace():
    n = 120
    p = pencil_1d(n)
    ks = [2, 3, 5, 8]
    V = np.stack([inertia.eigvec_1d(n, k) for k in ks], axis=1) @ start_block(4, 4, 1)
    theta, X = rr.rayleigh_ritz(p.A(), p.B(), V)
    np.testing.assert_allclose(theta, inertia.lambda_1d(n, ks), rtol=1e-11)
    np.testing.assert_allclose(X.T @ (p.B() @ X), np.eye(4), atol=1e-12)
    rho, rho_ax = rr.residuals(p.A(), p.B(), X, theta)
    assert rho.max() < 1e-9 and rho_ax.max() < 1e-9


def test_algorithm1_1d_matches_closed_form():
    n = 2000
    p = pencil_1d(n)
    lam = inertia.lambda_1d(n)
    gamma = 0.5 * (lam[19] + lam[20])
    s, w = poles.slrf_poles(2, 1.0, 0.01, gamma)
    res = subspace.subspace_iterate(p.A(), p.B(), s, w, gamma, start_block(n, 30, 2504), tol=1e-10)
    assert res.converged
    assert res.n_wanted == 20 == inertia.count_below_1d(n, gamma)
    np.testing.assert_allclose(res.theta[:20], lam[:20], rtol=1e-10)
    assert res.rho[:20].max() < 1e-8


def test_algorithm1_brute_force_small_2d():
    # n <= 200: Algorithm 1 against dense LAPACK eigh of the whole pencil.
    p = pencil_2d_q1(15, seed=7)          # n = 196
    lam = la.eigvalsh(p.A().toarray(), p.B().toarray())
    gamma = 0.5 * (lam[11] + lam[12])
    for rule in ("midpoint", "gauss_legendre"):
        s, w = poles.quadrature_poles(rule, 4, gamma)
        res = subspace.subspace_iterate(p.A(), p.B(), s, w, gamma, start_block(p.n, 18, 3), tol=1e-10)
        assert res.converged and res.n_wanted == 12
        np.testing.assert_allclose(res.theta[:12], lam[:12], rtol=1e-10)


# --------------------------------------------------------------------------
# lowest_eigs through its sparse (ARPACK shift-invert) branch, and the sparse
# inertia count on a node-block elasticity pencil.  These two functions write
# the stored 2D/3D spectra and counts that every full-size parity test uses.
#
# Tolerance: 1e-10 relative, the eigenvalue tolerance of the parity tests.
# FP64 rounding alone puts the lowest eigenvalues of these pencils ~1e-11 from
# the exact ones (dense LAPACK eigh and ARPACK differ by 3e-11 on the 2D
# pencil below; the 1D closed form sits 3e-11 from either), so a tighter gate
# would test rounding, not the routine.  A wrong mass operand, a wrong
# inverse operator or a dropped eigenvalue moves some lambda_k by at least
# the relative gap to its neighbour (>= 1e-4 here), far above the gate.
# --------------------------------------------------------------------------
def _check_lowest(p, k, lam_ref, lam, X):
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-10, atol=0)
    A, B = p.A(), p.B()
    # B-orthonormal eigenvectors (Section 2: x^T B x = 1) with small residuals
    np.testing.assert_allclose(X.T @ (B @ X), np.eye(k), atol=1e-10)
    # backward-error form of the residual: a backward-stable eigenpair has
    # ||A x - lambda B x|| <= c eps (||A|| + |lambda| ||B||) ||x||; a wrong
    # operand gives an O(1) residual
    R = A @ X - (B @ X) * lam[None, :]
    nA = abs(A).sum(axis=1).max()
    nB = abs(B).sum(axis=1).max()
    bound = 100 * np.finfo(float).eps * (nA + np.abs(lam) * nB) * np.linalg.norm(X, axis=0)
    assert np.all(np.linalg.norm(R, axis=0) <= bound), (np.linalg.norm(R, axis=0) / bound).max()
    # nothing dropped or doubled: the inertia count of A - gamma B at the gap
    # above lambda_k equals k (Sylvester's law, as in Algorithm 1's ENSURE)
    gamma = 0.5 * (lam_ref[k - 1] + lam_ref[k]) if len(lam_ref) > k else None
    return gamma


def test_lowest_eigs_sparse_branch_1d_closed_form():
    n, k = 5000, 30
    p = pencil_1d(n)
    lam, X = inertia.lowest_eigs(p.A(), p.B(), k, dense_limit=1000)   # forces ARPACK
    exact = inertia.lambda_1d(n)
    _check_lowest(p, k, exact[:k], lam, X)
    gamma = 0.5 * (exact[k - 1] + exact[k])
    assert inertia.count_below_1d(n, gamma) == k
    assert inertia.count_below_sparse(p.A(), p.B(), gamma) == k


def test_lowest_eigs_sparse_branch_2d_lognormal_against_dense():
    p = pencil_2d_q1(70, seed=17)          # n = 4761, lognormal coefficient
    k = 40
    ref = la.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True, subset_by_index=[0, k])
    lam, X = inertia.lowest_eigs(p.A(), p.B(), k, dense_limit=1000)
    _check_lowest(p, k, ref[:k], lam, X)
    gamma = 0.5 * (ref[k - 1] + ref[k])
    assert inertia.count_below_sparse(p.A(), p.B(), gamma) == k


def test_lowest_eigs_sparse_branch_3d_elasticity_against_dense():
    p = pencil_3d_elasticity(12, seed=19)  # 12^3 nodes, face x=0 clamped: n = 4752
    assert p.n == 4752
    k = 40
    ref = la.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True, subset_by_index=[0, k])
    lam, X = inertia.lowest_eigs(p.A(), p.B(), k, dense_limit=1000)
    _check_lowest(p, k, ref[:k], lam, X)


def test_sparse_count_on_elasticity_pencil_matches_dense():
    # node-block (3 dof per node) pencil: the case where diagonal-pivot-only
    # symmetric LU is most fragile; checked against a Bunch-Kaufman LDL^T.
    p = pencil_3d_elasticity(8, seed=23)   # n = 8*8*7*3 = 1344
    lam = la.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    for k in (1, 6, 25, 90, 400, 1000):
        gamma = 0.5 * (lam[k - 1] + lam[k])
        assert inertia.count_below_dense(p.A(), p.B(), gamma) == k
        assert inertia.count_below_sparse(p.A(), p.B(), gamma) == k


# --------------------------------------------------------------------------
# filter derivative and the shifted operator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 4, 8])
def test_separation_factor_of_the_midpoint_rule_closed_form(N):
    # The midpoint rule's filter is 1/(1 + ((x - c)/r)^(2N)) with c = r = gamma/2
    # (pinned above); its slope at x = gamma is -2N/(4r) = -N/gamma, so the
    # separation factor |Phi'(gamma)| (Definition 3.1) is N/gamma.
    for gamma in (1.0, 37.5):
        s, w = poles.quadrature_poles("midpoint", N, gamma)
        assert abs(poles.separation_factor(s, w, gamma) - N / gamma) < 1e-12 * N / gamma


@pytest.mark.parametrize("rule", ["gauss_legendre", "slrf"])
def test_filter_derivative_matches_central_differences(rule):
    s, w = poles.slrf_poles(4, 1.0, 0.01) if rule == "slrf" else poles.quadrature_poles(rule, 5, 1.0)
    x = np.linspace(-0.5, 3.0, 29)
    h = 1e-5
    fd = (poles.phi_real(x + h, s, w) - poles.phi_real(x - h, s, w)) / (2 * h)
    d = np.real(poles.dphi(x, s, w))
    np.testing.assert_allclose(d, fd, rtol=0, atol=1e-7 * max(1.0, np.abs(d).max()))


def test_shifted_product_on_closed_form_eigenvectors():
    # (A - sigma B) v_k = (lambda_k - sigma) B v_k for the 1D closed-form
    # eigenpairs, for complex shifts in both half planes and complex blocks.
    n = 64
    p = pencil_1d(n)
    ks = [1, 2, 9, 40]
    V = np.stack([inertia.eigvec_1d(n, k) for k in ks], axis=1)
    lam = inertia.lambda_1d(n, ks)
    coef = np.array([1.0, 0.5 - 2.0j, -1.5j, 3.0 + 1.0j])
    P = V * coef[None, :]
    BV = p.B() @ V
    for sigma in (120.0 + 35.0j, 3.0 - 80.0j, 0.0):
        Q = ofilt.shifted_product(p.A(), p.B(), sigma, P)
        expect = BV * ((lam - sigma) * coef)[None, :]
        np.testing.assert_allclose(Q, expect, rtol=0, atol=1e-9 * np.abs(expect).max())
