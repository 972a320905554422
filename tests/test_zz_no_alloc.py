"""The allocation-free Gram entry point (slrf_gram_noalloc).

Some callers may not allocate device memory themselves (their device memory
belongs to another allocator or a fixed pool, or they cannot take
cudaMalloc's implicit synchronisation); slrf_gram_noalloc serves them with a
static device scratch.  This file is collected last so that a failure here
leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import pencil_1d, start_block

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21618_gb300 import api as a
    return a


def _noalloc_gram(api, X, Y):
    m = X.shape[1]
    G = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
    st = api.load().slrf_gram_noalloc(X.shape[0], m, C.c_void_p(X.data_ptr()), X.stride(0),
                                      C.c_void_p(Y.data_ptr()), Y.stride(0), C.c_void_p(G.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == api.OK, api.load().slrf_noalloc_last_error()
    torch.cuda.synchronize()
    return G.cpu().numpy()


def test_noalloc_gram_matches_handle_gram_twice(api):
    # two calls in a row with different sizes and data: the second must not
    # see anything left in the shared scratch by the first
    for n, m, seed in [(20011, 150, 1), (3001, 77, 2)]:
        X = start_block(n, m, seed)
        Y = start_block(n, m, seed + 10)
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        h = api.Handle(pencil_1d(n))
        ref = h.gram(Xd, Yd).cpu().numpy()
        h.close()
        got = _noalloc_gram(api, Xd, Yd)
        tol = 1e-13 * np.abs(X).max() * np.abs(Y).max() * n
        assert np.abs(got - ref).max() <= tol
        assert np.abs(got - X.T @ Y).max() <= tol


def test_noalloc_gram_at_the_largest_accepted_size(api):
    # m = 724 is the largest m whose m x m partial product fits the scratch:
    # one K slice only, so the unsplit product path runs
    n, m = 20000, 724
    X = start_block(n, m, 31)
    Y = start_block(n, m, 32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    h = api.Handle(pencil_1d(n))
    ref = h.gram(Xd, Yd).cpu().numpy()
    h.close()
    tol = 1e-13 * np.abs(X).max() * np.abs(Y).max() * n
    for _ in range(2):
        got = _noalloc_gram(api, Xd, Yd)
        assert np.abs(got - ref).max() <= tol
        assert np.abs(got - X.T @ Y).max() <= tol


def test_noalloc_gram_rejects_m_beyond_scratch(api):
    m = 725
    X = torch.zeros((4, m), dtype=torch.float64, device="cuda")
    G = torch.zeros((1,), dtype=torch.float64, device="cuda")
    lib = api.load()
    st = lib.slrf_gram_noalloc(4, m, C.c_void_p(X.data_ptr()), m, C.c_void_p(X.data_ptr()), m,
                               C.c_void_p(G.data_ptr()), None)
    assert st == api.EINVAL
    assert b"exceeds the static scratch" in lib.slrf_noalloc_last_error()
