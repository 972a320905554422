"""Batched problems and the request server: every result equals the result of
the same problem solved alone (kernels reduce in a fixed order)."""
import time

import numpy as np
import pytest
import scipy.linalg as la

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


def _problems():
    out = []
    specs = [("1d", 600, 8), ("2d", 30, 12), ("2d", 41, 20), ("3d", 6, 10), ("1d", 1500, 15), ("2d", 25, 6)]
    for i, (kind, size, nev) in enumerate(specs):
        p = {"1d": lambda: pencil_1d(size), "2d": lambda: pencil_2d_q1(size, seed=30 + i),
             "3d": lambda: pencil_3d_elasticity(size, seed=40 + i)}[kind]()
        lam = la.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True, subset_by_index=[0, nev])
        gamma = 0.5 * (lam[nev - 1] + lam[nev])
        L = int(1.5 * nev)
        f = poles.slrf_poles(4, 1.0, 0.01, gamma)
        out.append((p, f, gamma, L, start_block(p.n, L, 100 + i), lam[:nev]))
    return out


def test_batch_matches_solo_bitwise(api):
    probs = _problems()
    solo = []
    for p, (s, w), gamma, L, V0, lam in probs:
        h = api.Handle(p)
        th, X, r, nc, st, _ = h.subspace_iterate(api.Filter(s, w), gamma, torch.from_numpy(V0).cuda())
        solo.append((th.cpu().numpy(), X.cpu().numpy(), st, nc))
        h.close()
    streams = [torch.cuda.Stream() for _ in probs]
    handles = [api.Handle(p, stream=st) for (p, *_), st in zip(probs, streams)]
    res = api.batch_iterate(handles, [api.Filter(*f) for _, f, *_ in probs], [g for _, _, g, *_ in probs],
                            [torch.from_numpy(V0).cuda() for *_, V0, _ in probs])
    for i, (th, X, r, nc, st, rep) in enumerate(res):
        assert st == solo[i][2] == api.OK
        assert nc == solo[i][3] == len(probs[i][5])
        np.testing.assert_array_equal(th.cpu().numpy(), solo[i][0])
        np.testing.assert_array_equal(X.cpu().numpy(), solo[i][1])
        np.testing.assert_allclose(th.cpu().numpy()[:nc], probs[i][5], rtol=1e-10)
    for h in handles:
        h.close()


def test_server_mix_matches_solo(api):
    probs = _problems()
    solo = []
    for p, (s, w), gamma, L, V0, lam in probs:
        h = api.Handle(p)
        th, X, r, nc, st, _ = h.subspace_iterate_host(api.Filter(s, w), gamma, V0)
        solo.append((th, X, st))
        h.close()
    srv0 = api.Server(n_workers=3)
    need = [srv0.bytes(srv0.request(p, api.Filter(*f), g, V0)) for p, f, g, L, V0, _ in probs]
    srv0.close()
    # budget admits roughly two of the largest requests at a time
    srv = api.Server(n_workers=3, mem_budget=int(2.2 * max(need)))
    tickets = []
    for i, (p, f, g, L, V0, _) in enumerate(probs):
        tickets.append(srv.submit(p, api.Filter(*f), g, V0))
        if i % 2 == 1:
            time.sleep(0.05)          # staggered arrivals while earlier ones run
    lats = []
    for i, t in enumerate(tickets):
        th, X, r, nc, st, rep, lat = srv.poll(t, wait=True)
        assert st == api.OK
        np.testing.assert_array_equal(th, solo[i][0])
        np.testing.assert_array_equal(X, solo[i][1])
        lats.append(lat)
    assert all(lt > 0 for lt in lats)
    assert srv.stats()["finished"] == len(probs)
    srv.close()


def test_server_rejects_request_beyond_budget(api):
    p = pencil_1d(500)
    srv = api.Server(n_workers=1, mem_budget=1 << 20)
    f = api.Filter(*poles.quadrature_poles("midpoint", 2, 1000.0))
    with pytest.raises(api.SlrfError):
        srv.submit(p, f, 1000.0, start_block(500, 8, 1))
    srv.close()
