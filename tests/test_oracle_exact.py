"""Pins for the oracle's exact solvers u = A^{-1} f (the plain definition of
the result): the sine-mode expansion against dense Cholesky of the assembled
operator, against the assembled operator's residual, and on single sine modes,
whose solution is the closed form v_m / lambda_m (Sec. 4 operator)."""
import numpy as np
import pytest

from oracle import exact, grid

CASES = [((5,), None), ((3, 4), None), ((4, 3), (0.7, 1.9)), ((2, 3, 2), (0.7, 1.9, 1.3)),
         ((2, 2, 1, 2), (1.0, 0.5, 2.0, 1.5)), ((2, 2, 2, 1, 2, 1), None)]


@pytest.mark.parametrize("levels,coeffs", CASES)
def test_sine_solve_equals_dense_cholesky(levels, coeffs):
    N = grid.num_unknowns(levels)
    f = np.random.default_rng(N).uniform(-1, 1, N)
    ud = exact.solve(levels, f, coeffs)
    us = exact.solve_sine(levels, f, coeffs)
    assert np.linalg.norm(us - ud) <= 1e-13 * np.linalg.norm(ud)


@pytest.mark.parametrize("levels,coeffs", [((6, 5, 4), (0.6, 1.3, 1.8)), ((5, 4, 3, 3, 2, 2), None)])
def test_sine_solve_residual(levels, coeffs):
    A = grid.stencil_matrix(levels, coeffs)
    f = np.random.default_rng(5).standard_normal(A.shape[0])
    u = exact.solve_sine(levels, f, coeffs)
    r = A @ u - f
    scale = abs(A) @ np.abs(u)
    assert np.all(np.abs(r) <= 1e-12 * scale.max())


@pytest.mark.parametrize("levels,coeffs", CASES + [((7, 6, 5), (0.9, 1.4, 0.6))])
def test_sine_solve_on_a_sine_mode(levels, coeffs):
    rng = np.random.default_rng(11)
    m = [int(rng.integers(1, 1 << l)) for l in levels]
    v = grid.sine_mode(levels, m)
    lam = grid.sine_eigenvalue(levels, m, coeffs)
    u = exact.solve_sine(levels, v, coeffs)
    assert np.linalg.norm(u - v / lam) <= 1e-13 * np.linalg.norm(v / lam)


def test_sine_eigenvalues_closed_form():
    levels, c = (3, 2), (1.5, 0.5)
    lam = exact.sine_eigenvalues(levels, c)
    for m1 in range(1, 8):
        for m2 in range(1, 4):
            assert np.isclose(lam[m1 - 1, m2 - 1], grid.sine_eigenvalue(levels, (m1, m2), c),
                              rtol=1e-15)


def test_adjoint_gradients_by_sine_solves_equal_direct():
    from oracle import adjoint
    levels, c = (4, 3, 3), np.array([0.8, 1.6, 1.1])
    N = grid.num_unknowns(levels)
    rng = np.random.default_rng(21)
    f, ut = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    u1, g1, c1 = adjoint.gradients(levels, f, ut, c)
    u2, g2, c2 = adjoint.gradients(levels, f, ut, c, method="sine")
    assert np.linalg.norm(g2 - g1) <= 1e-12 * np.linalg.norm(g1)
    assert np.allclose(c2, c1, rtol=1e-11, atol=0)
    # central differences of the exact loss, step 1e-4 (truncation ~1e-8 relative)
    for j in range(3):
        h = 1e-4 * c[j]
        cp, cm = c.copy(), c.copy()
        cp[j] += h
        cm[j] -= h
        up = exact.solve_sine(levels, f, cp)
        um = exact.solve_sine(levels, f, cm)
        fd = float(((up - um) * (up + um - 2 * ut)).sum()) / (2 * h)
        assert abs(fd - c2[j]) <= 1e-7 * abs(c2[j])
