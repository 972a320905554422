"""GPU parity of the individual hot-path steps against the FP64 oracle,
through the C ABI.  Sizes span several tiles and a ragged tail."""
import numpy as np
import pytest
import scipy.linalg as la

from oracle import filter as ofilt
from oracle import poles, rr
from workloads import pencil_1d, pencil_2d_q1, pencil_3d_elasticity, start_block

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21618_gb300 import api as a
    return a


def _cplx_block(n, N, m, ldp, seed):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, N, ldp), dtype=complex)
    P[:, :, :m] = rng.standard_normal((n, N, m)) + 1j * rng.standard_normal((n, N, m))
    return P


@pytest.mark.parametrize("prec,kernel", [("fp32", 1), ("fp32", 2), ("fp32", 3), ("fp32", 4), ("fp64", 1)])
@pytest.mark.parametrize("pencil,N,m,rows", [("2d", 3, 37, 0), ("3d", 2, 10, 0), ("1d", 1, 1, 0), ("2d", 9, 5, 0),
                                             ("2d", 2, 12, 1), ("2d", 2, 12, 3), ("2d", 4, 6, 4), ("3d", 1, 4, 2),
                                             ("2d", 4, 150, 0), ("3d", 3, 33, 0)])
def test_shifted_spmm_matches_oracle(api, prec, kernel, pencil, N, m, rows):
    # kernel 1: row groups gathered by every warp; 2: staged (bulk copies into
    # shared memory by a producer warp); 3: node blocks (3-dof pencils; others
    # run kernel 1); 4: SELL-C-sigma; each against the oracle's product
    p = {"2d": lambda: pencil_2d_q1(23, seed=4), "3d": lambda: pencil_3d_elasticity(5, seed=2),
         "1d": lambda: pencil_1d(77)}[pencil]()
    s, w = poles.quadrature_poles("gauss_legendre", N, 300.0)
    ldp = m + (m & 1)
    P = _cplx_block(p.n, N, m, ldp, 1)
    h = api.Handle(p, api.default_opts(spmm_rows=rows, spmm_kernel=kernel))
    f = api.Filter(s, w)
    cdt = np.complex64 if prec == "fp32" else np.complex128
    Pd = torch.from_numpy(P.astype(cdt).view(np.float32 if prec == "fp32" else np.float64).copy()).cuda()
    Q = torch.zeros_like(Pd)
    mu = torch.zeros(2 * N * m, dtype=Pd.dtype, device="cuda")
    h.shifted_spmm(f, Pd, m, ldp, prec=api.PREC_MIXED if prec == "fp32" else api.PREC_FP64, Q=Q, mu=mu)
    torch.cuda.synchronize()
    Qh = Q.cpu().numpy().view(cdt).reshape(p.n, N, ldp).astype(complex)
    muh = mu.cpu().numpy().view(cdt).reshape(N, m).astype(complex)
    tol = 2e-6 if prec == "fp32" else 1e-13
    A, B = p.A(), p.B()
    Pq = P.astype(cdt).astype(complex)   # the rounded input the kernel saw
    for j in range(N):
        ref = ofilt.shifted_product(A, B, s[j], Pq[:, j, :m])
        scale = np.abs(A).sum(axis=1).max() * np.abs(Pq).max() * (1 + abs(s[j]))
        assert np.abs(Qh[:, j, :m] - ref).max() <= tol * scale
        muref = np.sum(Pq[:, j, :m] * ref, axis=0)
        assert np.abs(muh[j] - muref).max() <= tol * scale * np.abs(Pq).max() * p.n


@pytest.mark.parametrize("pencil,rows,want", [("3d", 0, 3), ("3d", 2, 1), ("2d", 0, 1), ("1d", 0, 1)])
def test_node_block_kernel_runs_only_on_node_pencils(api, pencil, rows, want):
    # the node-block form exists for 3-dof pencils grouped by node; elsewhere
    # the request resolves to the row-group kernel, and the report says so
    p = {"2d": lambda: pencil_2d_q1(15, seed=4), "3d": lambda: pencil_3d_elasticity(4, seed=2),
         "1d": lambda: pencil_1d(90)}[pencil]()
    s, w = poles.quadrature_poles("gauss_legendre", 2, 300.0)
    h = api.Handle(p, api.default_opts(spmm_rows=rows, spmm_kernel=3, inner_tol=1e-4))
    V = torch.from_numpy(start_block(p.n, 4, 1)).cuda()
    U, st, rep = h.filter_apply(api.Filter(s, w), V)
    assert st == api.OK and rep.spmm_kernel == want


def test_node_block_kernel_on_graded_3d_pencil(api):
    # a larger elasticity pencil (several node groups per block, lognormal
    # stiffness), every column active, against the oracle's product
    p = pencil_3d_elasticity(9, seed=7)
    s, w = poles.slrf_poles(3, 1.0, 0.01, 40.0)
    N, m = len(s), 24
    P = _cplx_block(p.n, N, m, m, 5)
    out = {}
    for kernel in (1, 3):
        h = api.Handle(p, api.default_opts(spmm_kernel=kernel))
        Pd = torch.from_numpy(P.astype(np.complex64).view(np.float32).copy()).cuda()
        Q = torch.zeros_like(Pd)
        mu = torch.zeros(2 * N * m, dtype=Pd.dtype, device="cuda")
        h.shifted_spmm(api.Filter(s, w), Pd, m, m, prec=api.PREC_MIXED, Q=Q, mu=mu)
        torch.cuda.synchronize()
        out[kernel] = Q.cpu().numpy().view(np.complex64).reshape(p.n, N, m).astype(complex)
    A, B = p.A(), p.B()
    Pq = P.astype(np.complex64).astype(complex)
    for j in range(N):
        ref = ofilt.shifted_product(A, B, s[j], Pq[:, j])
        scale = np.abs(A).sum(axis=1).max() * np.abs(Pq).max() * (1 + abs(s[j]))
        for kernel in (1, 3):
            assert np.abs(out[kernel][:, j] - ref).max() <= 2e-6 * scale


@pytest.mark.parametrize("C,sigma", [(4, 1), (8, 7), (16, 256), (32, 1), (64, 10 ** 6)])
@pytest.mark.parametrize("pencil", ["2d", "3d", "1d"])
def test_sell_spmm_chunk_and_sorting_window(api, C, sigma, pencil):
    # SELL-C-sigma with chunk sizes that leave a ragged last chunk, sorting
    # windows from none (1) to the whole matrix; rows of unequal length (the
    # boundary rows of the 2D/3D pencils) make padded chunks
    p = {"2d": lambda: pencil_2d_q1(19, seed=6), "3d": lambda: pencil_3d_elasticity(4, seed=3),
         "1d": lambda: pencil_1d(131)}[pencil]()
    s, w = poles.quadrature_poles("gauss_legendre", 3, 200.0)
    N, m = len(s), 11
    ldp = m + 1
    P = _cplx_block(p.n, N, m, ldp, 4)
    h = api.Handle(p, api.default_opts(spmm_kernel=4, sell_c=C, sell_sigma=sigma))
    Pd = torch.from_numpy(P.astype(np.complex64).view(np.float32).copy()).cuda()
    Q = torch.zeros_like(Pd)
    mu = torch.zeros(2 * N * m, dtype=Pd.dtype, device="cuda")
    h.shifted_spmm(api.Filter(s, w), Pd, m, ldp, prec=api.PREC_MIXED, Q=Q, mu=mu)
    torch.cuda.synchronize()
    Qh = Q.cpu().numpy().view(np.complex64).reshape(p.n, N, ldp).astype(complex)
    muh = mu.cpu().numpy().view(np.complex64).reshape(N, m).astype(complex)
    A, B = p.A(), p.B()
    Pq = P.astype(np.complex64).astype(complex)
    for j in range(N):
        ref = ofilt.shifted_product(A, B, s[j], Pq[:, j, :m])
        scale = np.abs(A).sum(axis=1).max() * np.abs(Pq).max() * (1 + abs(s[j]))
        assert np.abs(Qh[:, j, :m] - ref).max() <= 2e-6 * scale
        assert np.all(Qh[:, j, m:] == 0)          # padding columns (zero in P) stay zero
        muref = np.sum(Pq[:, j, :m] * ref, axis=0)
        assert np.abs(muh[j] - muref).max() <= 2e-6 * scale * np.abs(Pq).max() * p.n


@pytest.mark.parametrize("m", [1, 30, 65])
def test_spmm_ab_matches_scipy(api, m):
    p = pencil_2d_q1(31, seed=8)
    X = start_block(p.n, m, 3)
    h = api.Handle(p)
    Xd = torch.from_numpy(X).cuda()
    Y, Z = h.spmm_ab(Xd)
    np.testing.assert_allclose(Y.cpu().numpy(), p.A() @ X, rtol=1e-13, atol=1e-13 * np.abs(p.A() @ X).max())
    np.testing.assert_allclose(Z.cpu().numpy(), p.B() @ X, rtol=1e-13, atol=1e-13 * np.abs(p.B() @ X).max())


@pytest.mark.parametrize("ozaki", [2, 1, 0])
@pytest.mark.parametrize("n,m", [(1000, 1), (5000, 64), (20011, 150), (3001, 77), (70000, 65), (4099, 300)])
def test_gram_matches_numpy(api, n, m, ozaki):
    p = pencil_1d(n)
    X = start_block(n, m, 1)
    Y = start_block(n, m, 2)
    h = api.Handle(p, api.default_opts(gram_ozaki=ozaki))
    G = h.gram(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).cpu().numpy()
    ref = X.T @ Y
    assert np.abs(G - ref).max() <= 1e-13 * np.abs(X).max() * np.abs(Y).max() * n


@pytest.mark.parametrize("ozaki", [2, 1, 0])
@pytest.mark.parametrize("n,k,m", [(1000, 1, 1), (5001, 150, 150), (20011, 31, 77), (3001, 300, 65), (777, 512, 40),
                                   (2049, 513, 33), (70000, 96, 150)])
def test_tall_product_matches_numpy(api, n, k, m, ozaki):
    # C = A B: rows of A graded over 20 decades (each row takes its own
    # exponent), columns of B over 10; k = 513 leaves the tensor-core form's
    # single 512-row K-slice and runs mma.sync
    rng = np.random.default_rng(n + k)
    A = rng.standard_normal((n, k)) * np.exp2(rng.integers(-33, 33, n))[:, None]
    B = rng.standard_normal((k, m)) * np.exp2(rng.integers(-16, 16, m))[None, :]
    h = api.Handle(pencil_1d(n), api.default_opts(gram_ozaki=ozaki))
    C = h.tall_product(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= 1e-13 * bound + 1e-300)


@pytest.mark.parametrize("ozaki", [2, 1])
def test_ozaki_gram_graded_columns(api, ozaki):
    # columns spanning 16 orders of magnitude, zero and subnormal-free tiny columns
    n, m = 9000, 40
    rng = np.random.default_rng(3)
    X = start_block(n, m, 4) * 10.0 ** rng.uniform(-8, 8, m)[None, :]
    Y = start_block(n, m, 5) * 10.0 ** rng.uniform(-8, 8, m)[None, :]
    X[:, 3] = 0.0
    h = api.Handle(pencil_1d(n), api.default_opts(gram_ozaki=ozaki))
    G = h.gram(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).cpu().numpy()
    ref = X.T @ Y
    bound = 1e-13 * np.abs(X).max(axis=0)[:, None] * np.abs(Y).max(axis=0)[None, :] * n
    assert np.all(np.abs(G - ref) <= bound)
    assert np.all(G[3] == 0.0)


def _sym_with_spectrum(m, lam, seed):
    Qr, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))
    return (Qr * lam[None, :]) @ Qr.T


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("case", ["random", "graded", "clusters", "tiny", "odd", "pairs", "wide", "m160"])
def test_syev_matches_lapack(api, mode, case):
    rng = np.random.default_rng(5)
    if case == "random":
        m = 150
        S = rng.standard_normal((m, m))
        S = S + S.T
    elif case == "graded":
        m = 120
        S = _sym_with_spectrum(m, np.geomspace(1.0, 3e3, m), 1)
    elif case == "clusters":
        m = 64
        lam = np.repeat(np.linspace(1, 50, 16), 4)          # exact multiplicity 4
        lam[::7] += 1e-9 * lam[::7]                           # and near-multiplicities
        S = _sym_with_spectrum(m, lam, 2)
    elif case == "tiny":
        m = 1
        S = np.array([[3.5]])
    elif case == "m160":
        # the largest size of the one-block FP32 stage (odd-pitch shared copy)
        m = 160
        S = rng.standard_normal((m, m))
        S = S + S.T
    elif case == "wide":
        # six decades, like the first projection of a random start block:
        # the FP32 stage leaves the low end unresolved, so large groups reach
        # the final FP64 Jacobi
        m = 150
        S = _sym_with_spectrum(m, np.geomspace(1.0, 1e6, m), 4)
    elif case == "pairs":
        # a spectrum like the projected problems': near-degenerate pairs at
        # relative gaps from 1e-3 down to 1e-12, graded magnitudes
        m = 150
        base = np.geomspace(1.0, 1e3, 75)
        gaps = np.geomspace(1e-3, 1e-12, 75)
        S = _sym_with_spectrum(m, np.sort(np.concatenate([base, base * (1 + gaps)])), 3)
    else:
        m = 33
        S = rng.standard_normal((m, m))
        S = S @ S.T
    p = pencil_1d(max(m, 8))
    h = api.Handle(p)
    h.set_opts(eig_refine=mode)
    lam, Q = h.syev(torch.from_numpy(np.ascontiguousarray(S)).cuda())
    lam = lam.cpu().numpy()
    Q = Q.cpu().numpy()
    ref = la.eigvalsh(S)
    nrm = np.linalg.norm(S, 2)
    assert np.abs(lam - ref).max() <= 1e-13 * nrm * max(1, m / 10)
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-13 * m
    assert np.abs(S @ Q - Q * lam[None, :]).max() <= 1e-12 * nrm


@pytest.mark.parametrize("m", [5, 24])
def test_rayleigh_ritz_matches_oracle(api, m):
    p = pencil_2d_q1(26, seed=12)
    A, B = p.A(), p.B()
    # a filtered-looking block: exact low eigenvectors mixed with noise
    lam, Xe = la.eigh(A.toarray(), B.toarray())
    U = Xe[:, :m] @ start_block(m, m, 1) + 1e-3 * start_block(p.n, m, 2)
    h = api.Handle(p)
    theta, X, resid = h.rayleigh_ritz(torch.from_numpy(U).cuda())
    theta_o, X_o = rr.rayleigh_ritz(A, B, U)
    rho_o, _ = rr.residuals(A, B, X_o, theta_o)
    np.testing.assert_allclose(theta.cpu().numpy(), theta_o, rtol=1e-11)
    np.testing.assert_allclose(resid.cpu().numpy(), rho_o, rtol=1e-6, atol=1e-13)
    Xh = X.cpu().numpy()
    np.testing.assert_allclose(Xh.T @ (B @ Xh), np.eye(m), atol=1e-11)
    # Ritz vectors agree up to sign (simple Ritz values)
    sgn = np.sign(np.sum(Xh * X_o, axis=0))
    np.testing.assert_allclose(Xh * sgn[None, :], X_o, atol=1e-8 * np.abs(X_o).max())


def test_rayleigh_ritz_survives_dependent_columns(api):
    # A repeated column (up to 1e-13) makes the B-Gram singular in FP64: the
    # unshifted Cholesky breaks down and the shifted Cholesky-QR3 fallback
    # must still return the exact Ritz values of the well-determined part.
    p = pencil_2d_q1(20, seed=3)
    A, B = p.A(), p.B()
    lam, Xe = la.eigh(A.toarray(), B.toarray())
    U = Xe[:, :6] @ start_block(6, 6, 4)
    U = np.concatenate([U, U[:, :1] + 1e-13 * start_block(p.n, 1, 5)], axis=1)
    h = api.Handle(p)
    theta, X, resid = h.rayleigh_ritz(torch.from_numpy(np.ascontiguousarray(U)).cuda())
    th = np.sort(theta.cpu().numpy())
    # six Ritz values reproduce lambda_1..6; the seventh comes from the noise direction
    hits = [np.min(np.abs(th - l)) / l for l in lam[:6]]
    assert max(hits) < 1e-9


@pytest.mark.parametrize("m,dup", [(80, 0), (150, 37), (97, 95), (40, 3)])
def test_rayleigh_ritz_cholesky_pivot_below_shift(api, m, dup):
    # a column repeated up to 1e-9 leaves a positive pivot far below the
    # shifted Cholesky-QR shift (column-scaled Gram: ~1e-18 against ~1e-8);
    # the first pass must treat it as a breakdown and refactor with the shift,
    # in the blocked form (m >= 64: first, middle or last block) and the
    # one-block form, and the Ritz values of the well-determined part stay
    # accurate
    p = pencil_2d_q1(20, seed=3)
    A, B = p.A(), p.B()
    lam, Xe = la.eigh(A.toarray(), B.toarray())
    U = Xe[:, :m - 1] @ start_block(m - 1, m - 1, 4)
    U = np.concatenate([U[:, :dup + 1], U[:, dup:dup + 1] + 1e-9 * start_block(p.n, 1, 5), U[:, dup + 1:]], axis=1)
    h = api.Handle(p)
    theta, X, resid = h.rayleigh_ritz(torch.from_numpy(np.ascontiguousarray(U)).cuda())
    th = np.sort(theta.cpu().numpy())
    hits = [np.min(np.abs(th - l)) / l for l in lam[:m - 1]]
    assert max(hits) < 1e-9


def test_fma_peak_is_plausible(api):
    # 152 SMs x 128 FP32 lanes x 2 flops x ~2 GHz ~ 80 TFLOP/s nominal; FP64
    # runs far slower on this part.  A broken timer or a dead-code-eliminated
    # loop reads far outside these ranges.
    f32 = api.fma_peak(api.PREC_MIXED)
    f64 = api.fma_peak(api.PREC_FP64)
    assert 20e12 < f32 < 120e12, f32
    assert 0.1e12 < f64 < 0.5 * f32, f64
