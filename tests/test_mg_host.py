"""CPU checks of host multigrid setup code that has no entry point of its
own, compiled here with g++ into a small harness (tests/mg_host_dump.cpp):

* the layouts of the finest level's fused transfers (mg_fused_layout): the
  "up" layout (groups of R fine rows, union of their coarse columns, R pairs
  per entry) and the "down" layout (coarse rows of F^T) must both hold
  exactly the products A P, B P, diag(a) P, diag(b) P of the library's
  prolongator P (exported by slrf_mg_transfer, multiplied here by scipy);
* the eigendecomposition of a level pencil (mg_level_eig), whose
  eigenvectors the coarsest solve applies: V^T A V = diag(lambda),
  V^T B V = I, lambda ascending and equal to LAPACK's."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from workloads import pencil_1d, pencil_2d_q1, pencil_3d_elasticity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_21618_gb300", "csrc")


@pytest.fixture(scope="module")
def api(lib):
    from paper_2503_21618_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def dump_tool(tmp_path_factory):
    gxx = shutil.which(os.environ.get("CXX", "g++"))
    if gxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("mgh") / "mg_host_dump")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "mg_host_dump.cpp"),
                    os.path.join(CSRC, "mg_setup.cpp"), os.path.join(CSRC, "host_pool.cpp"), "-lpthread", "-o", exe],
                   check=True)
    return exe


def _write_pencil(p, d):
    np.asarray([p.n, len(p.col_idx)], np.int64).tofile(os.path.join(d, "hdr.bin"))
    np.asarray(p.row_ptr, np.int32).tofile(os.path.join(d, "rp.bin"))
    np.asarray(p.col_idx, np.int32).tofile(os.path.join(d, "ci.bin"))
    np.asarray(p.a_val, np.float64).tofile(os.path.join(d, "a.bin"))
    np.asarray(p.b_val, np.float64).tofile(os.path.join(d, "b.bin"))


def _dump(exe, p, block, R, d):
    _write_pencil(p, d)
    subprocess.run([exe, d, "layout", str(block), str(R)], check=True)
    rd = lambda name, dt: np.fromfile(os.path.join(d, name), dtype=dt)  # noqa: E731
    n1, nu, nd = rd("out_hdr.bin", np.int64)
    return (int(n1), rd("up_ptr.bin", np.int32), rd("up_col.bin", np.int32), rd("down_ptr.bin", np.int32),
            rd("down_col.bin", np.int32), rd("q.bin", np.float64).reshape(-1, 4), int(nu), int(nd))


@pytest.mark.parametrize("case", ["2d", "1d_odd", "3d_blocks"])
def test_fused_layouts_hold_the_products_of_p(api, dump_tool, tmp_path, case):
    if case == "2d":
        p, block, R, opts = pencil_2d_q1(22, seed=9), 1, 2, api.default_opts()
    elif case == "1d_odd":
        p, block, R, opts = pencil_1d(401), 1, 2, api.default_opts()      # ragged last group
    else:
        p, block, R, opts = pencil_3d_elasticity(5), 3, 3, api.default_opts(mg_coarse=30)
    n1, up_ptr, up_col, down_ptr, down_col, q, nu, nd = _dump(dump_tool, p, block, R, str(tmp_path))
    (ptr, col, val, nr, nc), _ = api.mg_transfer(p, 0, opts)
    assert nc == n1 and nr == p.n
    P = sp.csr_matrix((val, col, ptr), shape=(nr, nc))
    A, B = p.A().tocsr(), p.B().tocsr()
    want = [(A @ P).toarray(), (B @ P).toarray(), (sp.diags(A.diagonal()) @ P).toarray(),
            (sp.diags(B.diagonal()) @ P).toarray()]
    scale = [np.abs(w).max() for w in want]
    n, ng = p.n, (p.n + R - 1) // R
    # up layout: sorted unique columns per group; R pairs per entry, zero past the last row
    assert len(up_ptr) == ng + 1 and up_ptr[0] == 0 and up_ptr[-1] == nu and np.all(np.diff(up_ptr) >= 0)
    assert q.shape[0] == nu * R + nd
    got = [np.zeros((n, n1)) for _ in range(4)]
    for g in range(ng):
        cols = up_col[up_ptr[g]:up_ptr[g + 1]]
        assert np.all(np.diff(cols) > 0)
        for e in range(up_ptr[g], up_ptr[g + 1]):
            for r in range(R):
                row = g * R + r
                if row >= n:
                    assert np.all(q[e * R + r] == 0)
                    continue
                for t in range(4):
                    got[t][row, up_col[e]] = q[e * R + r, t]
    for t in range(4):
        np.testing.assert_allclose(got[t], want[t], rtol=0, atol=1e-13 * scale[t])
    # down layout: F^T by coarse rows, ascending fine columns, the same values
    assert len(down_ptr) == n1 + 1 and down_ptr[-1] == nd
    got = [np.zeros((n, n1)) for _ in range(4)]
    qd = q[nu * R:]
    for c in range(n1):
        rows = down_col[down_ptr[c]:down_ptr[c + 1]]
        assert np.all(np.diff(rows) > 0)
        for e in range(down_ptr[c], down_ptr[c + 1]):
            for t in range(4):
                got[t][down_col[e], c] = qd[e, t]
    for t in range(4):
        np.testing.assert_allclose(got[t], want[t], rtol=0, atol=1e-13 * scale[t])


@pytest.mark.parametrize("case", ["226", "725"])
def test_level_eigendecomposition(dump_tool, tmp_path, case):
    # 226: the coarsest level of a 2D hierarchy (one thread); 725: the level
    # a deep shift solves exactly (the threaded path)
    if case == "226":
        p, level = pencil_2d_q1(120, seed=7), 2
    else:
        p, level = pencil_2d_q1(80, seed=7), 1
    d = str(tmp_path)
    _write_pencil(p, d)
    subprocess.run([dump_tool, d, "eig", "1", str(level)], check=True)
    lam = np.fromfile(os.path.join(d, "lam.bin"))
    m = lam.size
    A = np.fromfile(os.path.join(d, "Ad.bin")).reshape(m, m)
    B = np.fromfile(os.path.join(d, "Bd.bin")).reshape(m, m)
    V = np.fromfile(os.path.join(d, "V.bin")).reshape(m, m)
    assert np.all(np.diff(lam) >= 0)
    np.testing.assert_allclose(lam, sla.eigh(A, B, eigvals_only=True), rtol=1e-10)
    np.testing.assert_allclose(V.T @ A @ V, np.diag(lam), rtol=0, atol=1e-13 * np.abs(lam).max())
    np.testing.assert_allclose(V.T @ B @ V, np.eye(m), rtol=0, atol=1e-13)


def test_setup_does_not_depend_on_the_thread_count(dump_tool, tmp_path):
    # power iteration, strength graph, row products, level eigensolver and
    # layouts on 1, 4 and 16 host threads (every step of the finest level
    # above the size at which it takes threads): byte-identical outputs
    p = pencil_2d_q1(160, seed=7)
    outs = {}
    for nt in (1, 4, 16):
        d = str(tmp_path / f"t{nt}")
        os.makedirs(d)
        _write_pencil(p, d)
        env = dict(os.environ, SLRF_HOST_THREADS=str(nt))
        subprocess.run([dump_tool, d, "eig", "1", "2"], check=True, env=env)
        subprocess.run([dump_tool, d, "layout", "1", "2"], check=True, env=env)
        outs[nt] = {f: open(os.path.join(d, f), "rb").read()
                    for f in ("lam.bin", "V.bin", "Ad.bin", "Bd.bin", "up_col.bin", "down_col.bin", "q.bin")}
    for nt in (4, 16):
        for f in outs[1]:
            assert outs[1][f] == outs[nt][f], (nt, f)


def _two_grid_factor(A, P, omega):
    # spectral radius of S (I - P A_c^{-1} P^T A) S, S = I - omega D^{-1} A
    # (one damped Jacobi sweep before and after an exact coarse correction)
    A = A.toarray()
    n = A.shape[0]
    S = np.eye(n) - omega * A / np.diag(A)[:, None]
    P = P.toarray()
    Ac = P.T @ A @ P
    C = np.eye(n) - P @ np.linalg.solve(Ac, P.T @ A)
    return float(np.abs(np.linalg.eigvals(S @ C @ S)).max())


def test_rigid_body_near_null_space(dump_tool, tmp_path):
    # With the six rigid-body modes Bn as near-null space (block 3), each
    # aggregate's tentative block is Q of the QR of its rows, so T Bc = Bn
    # with Bc the stacked R factors, and the smoothed prolongator satisfies
    # P Bc = Bn - w D^{-1} A Bn (w = 4 / (3 rho)); the next level is the
    # Galerkin pencil with 6 dofs per node; and a two-grid cycle converges
    # faster than with translations alone.
    from workloads import rigid_body_modes
    p = pencil_3d_elasticity(7, seed=11)             # n = 882
    Bn = rigid_body_modes(p)
    out = {}
    for k in (6, 0):
        d = str(tmp_path / f"k{k}")
        os.makedirs(d)
        _write_pencil(p, d)
        np.asarray(Bn, np.float64).tofile(os.path.join(d, "nul.bin"))
        subprocess.run([dump_tool, d, "nullspace", "3", str(k)], check=True)
        rd = lambda name, dt: np.fromfile(os.path.join(d, name), dtype=dt)  # noqa: E731
        sizes = rd("sizes.bin", np.int64)
        P = sp.csr_matrix((rd("p_val.bin", np.float64), rd("p_col.bin", np.int32), rd("p_ptr.bin", np.int32)),
                          shape=(p.n, int(sizes[1])))
        L1 = sp.csr_matrix((rd("l1_a.bin", np.float64), rd("l1_col.bin", np.int32), rd("l1_ptr.bin", np.int32)),
                           shape=(int(sizes[1]),) * 2)
        B1 = sp.csr_matrix((rd("l1_b.bin", np.float64), rd("l1_col.bin", np.int32), rd("l1_ptr.bin", np.int32)),
                           shape=(int(sizes[1]),) * 2)
        out[k] = dict(sizes=sizes, P=P, A1=L1, B1=B1, rho=float(rd("rho0.bin", np.float64)[0]),
                      diag=rd("diag0.bin", np.float64), nul=rd("l1_nul.bin", np.float64))
    r = out[6]
    nc = int(r["sizes"][1])
    assert nc % 6 == 0 and r["nul"].size == nc * 6
    Bc = r["nul"].reshape(nc, 6)
    A, M = p.A(), p.B()
    w = 4.0 / (3.0 * r["rho"])
    rhs = Bn - w * (A @ Bn) / r["diag"][:, None]
    np.testing.assert_allclose(r["P"] @ Bc, rhs, rtol=0, atol=1e-9 * np.abs(rhs).max())
    Ac = (r["P"].T @ A @ r["P"]).toarray()
    Mc = (r["P"].T @ M @ r["P"]).toarray()
    np.testing.assert_allclose(r["A1"].toarray(), Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())
    np.testing.assert_allclose(r["B1"].toarray(), Mc, rtol=0, atol=1e-12 * np.abs(Mc).max())
    # smoother damping 1/rho(D^-1 A), the same for both hierarchies
    rho_rbm = _two_grid_factor(A, r["P"], 1.0 / r["rho"])
    rho_trn = _two_grid_factor(A, out[0]["P"], 1.0 / r["rho"])
    # (measured 0.87 against 0.96: ~3.8 times the convergence rate per cycle)
    assert rho_trn < 1.0 and np.log(rho_rbm) < 2.0 * np.log(rho_trn), (rho_rbm, rho_trn)


def test_near_null_space_with_a_rank_deficient_block(dump_tool, tmp_path):
    # A chain of 3-dof nodes on the x axis: the rotation about x vanishes
    # (a zero column) and the other modes leave every aggregate's block one
    # short of rank 6, so each block of T is completed with a unit vector.
    # The hierarchy still builds, reproduces the near-null space through the
    # R factors (P B_c = B_n - w D^{-1} A B_n) and has a positive diagonal.
    nn = 300
    L1 = sp.diags([-np.ones(nn - 1), 2.0 * np.ones(nn), -np.ones(nn - 1)], [-1, 0, 1])
    M1 = sp.diags([np.ones(nn - 1), 4.0 * np.ones(nn), np.ones(nn - 1)], [-1, 0, 1]) / 6.0
    C = np.array([[2.0, 0.3, 0.1], [0.3, 1.5, 0.2], [0.1, 0.2, 1.0]])
    A = sp.kron(L1, C).tocsr()
    A.sort_indices()
    rows = np.repeat(np.arange(3 * nn), np.diff(A.indptr))
    b_val = sp.kron(M1, np.eye(3)).toarray()[rows, A.indices]    # B on A's (union) pattern
    from workloads import Pencil
    p = Pencil(n=3 * nn, row_ptr=A.indptr.astype(np.int32), col_idx=A.indices.astype(np.int32),
               a_val=A.data.astype(np.float64), b_val=b_val.astype(np.float64))
    x = np.arange(nn) / nn - 0.5
    Bn = np.zeros((3 * nn, 6))
    for c in range(3):
        Bn[c::3, c] = 1.0
    Bn[2::3, 4] = -x               # rotation about y on the x axis
    Bn[1::3, 5] = x                # rotation about z; column 3 (about x) stays zero
    d = str(tmp_path)
    _write_pencil(p, d)
    Bn.tofile(os.path.join(d, "nul.bin"))
    subprocess.run([dump_tool, d, "nullspace", "3", "6"], check=True)
    rd = lambda name, dt: np.fromfile(os.path.join(d, name), dtype=dt)  # noqa: E731
    sizes = rd("sizes.bin", np.int64)
    nc = int(sizes[1])
    assert nc % 6 == 0 and nc < 3 * nn
    P = sp.csr_matrix((rd("p_val.bin", np.float64), rd("p_col.bin", np.int32), rd("p_ptr.bin", np.int32)),
                      shape=(3 * nn, nc))
    Bc = rd("l1_nul.bin", np.float64).reshape(nc, 6)
    w = 4.0 / (3.0 * float(rd("rho0.bin", np.float64)[0]))
    rhs = Bn - w * (A @ Bn) / rd("diag0.bin", np.float64)[:, None]
    np.testing.assert_allclose(P @ Bc, rhs, rtol=0, atol=1e-9 * np.abs(rhs).max())
    assert np.abs(Bc[:, 3]).max() == 0.0          # the zero mode stays zero on the next level
    A1 = sp.csr_matrix((rd("l1_a.bin", np.float64), rd("l1_col.bin", np.int32), rd("l1_ptr.bin", np.int32)),
                       shape=(nc, nc))
    assert (A1.diagonal() > 0).all()


def _vcycle(As, Bs, Ps, s, omega=4.0 / 3.0, exact_max=400):
    # V(1,1) cycle for A - s B: damped Jacobi (omega / rho(D_l^-1 A_l)) on each
    # level down to the first with at most exact_max unknowns, solved exactly
    import scipy.sparse.linalg as spla
    c = next((l for l in range(1, len(As)) if As[l].shape[0] <= exact_max), len(As) - 1)
    Ks = [(As[l] - s * Bs[l]).tocsr() for l in range(c + 1)]
    Ds = []
    for l in range(c):
        Dinv = sp.diags(1.0 / As[l].diagonal())
        rho = abs(spla.eigs(Dinv @ As[l], k=1, which="LM", return_eigenvectors=False)[0])
        Ds.append((omega / rho) / Ks[l].diagonal())
    lu = spla.splu(Ks[c].tocsc())

    def cyc(l, r):
        if l == c:
            return lu.solve(r)
        z = Ds[l] * r
        z = z + Ps[l] @ cyc(l + 1, Ps[l].T @ (r - Ks[l] @ z))
        return z + Ds[l] * (r - Ks[l] @ z)
    return lambda r: cyc(0, r)


def _cocg_iterations(K, b, prec, tol=1e-5, maxit=2000):
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    d = z.copy()
    rho = r @ z
    b0 = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        q = K @ d
        al = rho / (d @ q)
        x += al * d
        r -= al * q
        if np.linalg.norm(r) <= tol * b0:
            return it
        z = prec(r)
        rn = r @ z
        d = z + (rn / rho) * d
        rho = rn
    return maxit


def test_rigid_body_cycle_for_the_shifted_systems(dump_tool, tmp_path):
    # COCG iterations for the complex-shifted systems (A - sigma_j B) y = B v
    # of the four SLRF poles of an interval holding 12 modes of an elasticity
    # cube, preconditioned by a V(1,1) cycle on each hierarchy: the rigid-body
    # hierarchy needs fewer iterations than translations alone at every pole
    # (both far fewer than Jacobi; measured 18-19 against 32-35 and 100-108).
    import scipy.sparse.linalg as spla
    from oracle import poles as opoles
    from workloads import rigid_body_modes
    p = pencil_3d_elasticity(9, seed=4)              # n = 1 944
    A, M = p.A().tocsr(), p.B().tocsr()
    lam = np.sort(spla.eigsh(A, k=14, M=M, sigma=0.0, return_eigenvectors=False))
    gamma = 0.5 * (lam[11] + lam[12])
    sig, _ = opoles.slrf_poles(4, 1.0, 0.01, gamma)
    hier = {}
    for k in (0, 6):
        d = str(tmp_path / f"h{k}")
        os.makedirs(d)
        _write_pencil(p, d)
        rigid_body_modes(p).tofile(os.path.join(d, "nul.bin"))
        subprocess.run([dump_tool, d, "nullspace", "3", str(k)], check=True)
        sizes = np.fromfile(os.path.join(d, "sizes.bin"), np.int64)
        Ps = []
        for l in range(len(sizes) - 1):
            rd = lambda name, dt: np.fromfile(os.path.join(d, f"p{l}_{name}.bin"), dtype=dt)  # noqa: E731
            Ps.append(sp.csr_matrix((rd("val", np.float64), rd("col", np.int32), rd("ptr", np.int32)),
                                    shape=(int(sizes[l]), int(sizes[l + 1]))))
        As, Bs = [A], [M]
        for P in Ps:
            As.append((P.T @ As[-1] @ P).tocsr())
            Bs.append((P.T @ Bs[-1] @ P).tocsr())
        hier[k] = (As, Bs, Ps)
    b = (M @ np.random.default_rng(9).standard_normal(p.n)).astype(complex)
    for s in sig:
        K = (A - s * M).tocsr()
        it = {k: _cocg_iterations(K, b, _vcycle(*hier[k], s)) for k in (0, 6)}
        it_j = _cocg_iterations(K, b, lambda r, dk=1.0 / K.diagonal(): dk * r)
        assert it[6] < it[0] < it_j, (s, it, it_j)


def test_near_null_space_through_the_c_abi(api):
    # slrf_mg_transfer / slrf_mg_describe with opts.mg_near_null: level 0's P
    # has 6 columns per aggregate and spans B_n - w D^{-1} A B_n; invalid
    # near-null options are rejected.
    from workloads import rigid_body_modes
    p = pencil_3d_elasticity(7, seed=11)
    Bn = rigid_body_modes(p)
    o = api.default_opts(precond=2, mg_near_null=Bn)
    assert o.mg_n_null == 6
    (ptr, col, val, nr, nc), rho = api.mg_transfer(p, 0, o)
    assert nr == p.n and nc % 6 == 0
    P = sp.csr_matrix((val, col, ptr), shape=(nr, nc))
    A = p.A()
    rhs = Bn - (4.0 / (3.0 * rho)) * (A @ Bn) / A.diagonal()[:, None]
    y, *_ = np.linalg.lstsq(P.toarray(), rhs, rcond=None)
    assert np.abs(P @ y - rhs).max() < 1e-9 * np.abs(rhs).max()
    d = api.mg_describe(p, o)
    assert d["levels"][1] == nc
    assert api.mg_describe(p, api.default_opts(precond=2))["levels"][1] != nc   # translations: 3 per aggregate
    bad = Bn.copy()
    bad[5, 2] = np.nan
    for opts in (api.default_opts(precond=2, mg_near_null=bad), api.default_opts(precond=2, mg_n_null=6),
                 api.default_opts(precond=2, mg_n_null=17, mg_near_null=np.zeros((p.n, 17)))):
        with pytest.raises(RuntimeError):
            api.mg_transfer(p, 0, opts)
