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
