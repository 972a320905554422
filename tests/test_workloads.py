"""Pins for the synthetic FE pencils (symmetry, definiteness, element facts)."""
import numpy as np
import scipy.linalg as la

from workloads import fe


def test_q1_unit_stiffness_is_tensor_form():
    # Bilinear elements: K2 = K1 (x) M1 + M1 (x) K1, mass M1 (x) M1.
    m = 7
    p1 = fe.pencil_1d(m - 1)
    K1 = p1.A().toarray()
    M1 = p1.B().toarray()
    p2 = fe.pencil_2d_q1(m, seed=None)
    np.testing.assert_allclose(p2.A().toarray(), np.kron(K1, M1) + np.kron(M1, K1), atol=1e-13)
    np.testing.assert_allclose(p2.B().toarray(), np.kron(M1, M1), atol=1e-16)


def test_hex8_element_rigid_modes_and_mass():
    h = 0.25
    K, M = fe.hex8_elasticity_element(h, nu=0.3, rho=2.0)
    ev = la.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6      # 3 translations + 3 rotations
    assert ev.min() > -1e-10 * ev.max()
    # total mass per direction = rho * h^3
    for comp in range(3):
        np.testing.assert_allclose(M[comp::3, comp::3].sum(), 2.0 * h ** 3, rtol=1e-14)
    np.testing.assert_allclose(K, K.T, atol=0)


def test_3d_pencil_spd_and_sizes():
    p = fe.pencil_3d_elasticity(4, seed=1)
    assert p.n == 3 * 3 * 4 * 4
    A = p.A().toarray()
    B = p.B().toarray()
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_array_equal(B, B.T)
    assert la.eigvalsh(A).min() > 0
    assert la.eigvalsh(B).min() > 0


def test_config_sizes():
    assert fe.pencil_2d_q1(300).nnz == 801025
    p = fe.pencil_2d_q1(20, seed=4)
    assert p.n == 19 * 19
    assert np.all(np.diff(p.row_ptr) <= 9)


def test_generators_are_seeded():
    a = fe.pencil_2d_q1(12, seed=5)
    b = fe.pencil_2d_q1(12, seed=5)
    c = fe.pencil_2d_q1(12, seed=6)
    np.testing.assert_array_equal(a.a_val, b.a_val)
    assert not np.array_equal(a.a_val, c.a_val)
    np.testing.assert_array_equal(fe.start_block(10, 3, 1), fe.start_block(10, 3, 1))


def test_rigid_body_modes_are_annihilated_away_from_the_clamp():
    # A B = 0 on every row whose element neighbourhood avoids the clamped face
    # (x = 0): translations and rotations strain no element; B has rank 6.
    from workloads import pencil_3d_elasticity, rigid_body_modes
    p = pencil_3d_elasticity(6, seed=3)
    B = rigid_body_modes(p)
    assert B.shape == (p.n, 6)
    assert np.linalg.matrix_rank(B) == 6
    node = np.arange(p.n // 3)
    far = np.repeat(node % (p.meta["p"] - 1) + 1 >= 2, 3)
    r = p.A() @ B
    assert np.abs(r[far]).max() < 1e-12 * np.abs(p.a_val).max()
    assert np.abs(r[~far]).max() > 1e-3 * np.abs(p.a_val).max()   # the clamp breaks it
