"""Pins for the oracle's grid and finite-difference operator (eq. dof; Sec. 4)."""
import numpy as np
import pytest

from oracle import grid


def test_dof_formula():
    assert grid.num_unknowns((6, 6)) == 3969
    assert grid.num_unknowns((10, 5, 3)) == 1023 * 31 * 7 == 221991
    assert grid.num_unknowns((5, 4, 3, 3, 2, 2)) == 205065
    assert grid.num_unknowns((8, 8, 6)) == 4096575


@pytest.mark.parametrize("levels,coeffs", [((5,), None), ((3, 4), None), ((3, 2, 2), None),
                                           ((2, 3, 2), (0.7, 1.9, 1.3)),
                                           ((2, 2, 1, 2), (1.0, 0.5, 2.0, 1.5))])
def test_sine_modes_are_eigenvectors(levels, coeffs):
    A = grid.stencil_matrix(levels, coeffs)
    rng = np.random.default_rng(3)
    for _ in range(5):
        m = [int(rng.integers(1, (1 << l))) for l in levels]
        v = grid.sine_mode(levels, m)
        lam = grid.sine_eigenvalue(levels, m, coeffs)
        assert np.linalg.norm(A @ v - lam * v) <= 1e-12 * lam * np.linalg.norm(v)


def test_level_one_axes_give_reaction_term():
    # Sec. 4.2: l = (L, 1, ..., 1) is the 1-D operator plus 8 (d - 1) I.
    L = 6
    for d in (2, 3, 4):
        A = grid.stencil_matrix((L,) + (1,) * (d - 1)).toarray()
        A1 = grid.stencil_matrix((L,)).toarray()
        assert np.array_equal(A, A1 + 8.0 * (d - 1) * np.eye(A1.shape[0]))


def test_one_dimensional_operator_by_hand():
    # h = 1/8: 64 * tridiag(-1, 2, -1)
    A = grid.stencil_matrix((3,)).toarray()
    T = 2 * np.eye(7) - np.eye(7, k=1) - np.eye(7, k=-1)
    assert np.array_equal(A, 64.0 * T)


def test_symmetric_positive_definite():
    A = grid.stencil_matrix((3, 2, 2), (1.0, 2.0, 0.5)).toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
