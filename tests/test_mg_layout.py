"""CPU check of the host logic that lays out the finest multigrid level's
fused transfers (mg_fused_layout, host C++ compiled here with g++): the
"up" layout (groups of R fine rows, union of their coarse columns, R pairs
per entry) and the "down" layout (coarse rows of F^T) must both hold exactly
the products A P, B P, diag(a) P, diag(b) P of the library's prolongator P
(exported by slrf_mg_transfer, multiplied here by scipy)."""
import os
import shutil
import subprocess

import numpy as np
import pytest
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
    exe = str(tmp_path_factory.mktemp("mgl") / "mg_layout_dump")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "mg_layout_dump.cpp"),
                    os.path.join(CSRC, "mg_setup.cpp"), "-lpthread", "-o", exe], check=True)
    return exe


def _dump(exe, p, block, R, d):
    np.asarray([p.n, len(p.col_idx)], np.int64).tofile(os.path.join(d, "hdr.bin"))
    np.asarray(p.row_ptr, np.int32).tofile(os.path.join(d, "rp.bin"))
    np.asarray(p.col_idx, np.int32).tofile(os.path.join(d, "ci.bin"))
    np.asarray(p.a_val, np.float64).tofile(os.path.join(d, "a.bin"))
    np.asarray(p.b_val, np.float64).tofile(os.path.join(d, "b.bin"))
    subprocess.run([exe, d, str(block), str(R)], check=True)
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
