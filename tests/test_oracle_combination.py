"""Pins of the oracle's combination formula (eq. combi) and of the Poisson test
problem of the combination-technique study (Sec. 4.3).

Expected values come from the mathematics: the interpolant reproduces nodal
values and every function that is multilinear on each cell of its grid; the
level-1 hat product lies in every subgrid's space, so the combination returns it
exactly (the coefficients times the layer sizes sum to one); the combined
interpolant of a smooth product function converges at second order in h_L up
to the logarithmic factor; the discrete solutions of the test problem converge
to u(x) = ||x||_2 prod sin(pi x_i) at second order.
"""
from math import comb

import numpy as np
import pytest

from oracle import combi, exact, grid
from paper_2110_11211_gb300 import inputs


def hat1(x):
    """The level-1 hat function 1 - |2x - 1| on [0, 1]."""
    return 1.0 - np.abs(2.0 * x - 1.0)


def nodal(levels, fn):
    K = grid.lex_coords(levels).astype(np.float64)
    X = K / np.array([float(1 << l) for l in levels])
    return fn(X)


def test_interpolant_reproduces_nodes_and_boundary():
    levels = (3, 2, 4)
    v = inputs.uniform(5, grid.num_unknowns(levels))
    K = grid.lex_coords(levels).astype(np.float64)
    X = K / np.array([8.0, 4.0, 16.0])
    assert np.allclose(combi.interpolate(levels, v, X), v, rtol=0, atol=1e-15)
    edge = np.array([[0.0, 0.5, 0.5], [1.0, 0.25, 0.5], [0.5, 1.0, 0.0625]])
    assert np.all(combi.interpolate(levels, v, edge) == 0.0)


def test_interpolant_exact_for_cellwise_multilinear():
    """prod_j hat1(x_j) is linear in every x_j on each cell of a level >= 1 grid."""
    fn = lambda X: np.prod(hat1(X), axis=1)
    pts = inputs.unit_points(6, 300, 3)
    for levels in [(1, 1, 1), (2, 1, 3), (4, 3, 2)]:
        got = combi.interpolate(levels, nodal(levels, fn), pts)
        assert np.allclose(got, fn(pts), rtol=0, atol=1e-14)


def test_interpolant_of_a_bilinear_cell_function():
    """On level (1, 1) the only interior node is the centre; the interpolant
    is hat1(x) hat1(y) scaled by the nodal value."""
    pts = inputs.unit_points(7, 50, 2)
    got = combi.interpolate((1, 1), np.array([2.5]), pts)
    assert np.allclose(got, 2.5 * hat1(pts[:, 0]) * hat1(pts[:, 1]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("d,L", [(2, 4), (3, 3), (4, 3)])
def test_combination_reproduces_the_level_one_hat(d, L):
    # the coefficients times the layer sizes sum to one
    assert sum((-1) ** i * comb(d - 1, i) * comb(L + d - 2 - i, d - 1) for i in range(d)) == 1
    fn = lambda X: np.prod(hat1(X), axis=1)
    pts = inputs.unit_points(8, 200, d)
    sols = {lv: nodal(lv, fn) for lv, _ in combi.full_layer_set(d, L)}
    assert np.allclose(combi.combine(d, L, sols, pts), fn(pts), rtol=0, atol=1e-13)


def test_full_layer_set_matches_the_counts():
    d, L = 4, 6
    s = combi.full_layer_set(d, L)
    for i in range(d):
        lv = [l for l, w in s if sum(l) == L + d - 1 - i]
        assert len(lv) == combi.layer_count(d, L, i)
        assert all(w == (-1) ** i * comb(d - 1, i) for l, w in s if sum(l) == L + d - 1 - i)


def test_combined_interpolant_converges_at_second_order():
    """Sparse-grid interpolation error of a smooth product function:
    O(h_L^2 L^{d-1}); the error ratio per level stays near 4 (above 3)."""
    d = 2
    fn = lambda X: np.prod(np.sin(np.pi * X), axis=1) * np.exp(X[:, 0])
    pts = inputs.unit_points(9, 400, d)
    errs = []
    for L in (4, 5, 6, 7):
        sols = {lv: nodal(lv, fn) for lv, _ in combi.full_layer_set(d, L)}
        errs.append(np.abs(combi.combine(d, L, sols, pts) - fn(pts)).max())
    for a, b in zip(errs, errs[1:]):
        assert a / b > 3.0, errs


def test_poisson_test_problem_rhs_second_order():
    """The discrete solutions of A u_h = f on full grids converge to the Sec. 4.3
    solution at second order: a dropped term or a wrong sign in f breaks this."""
    for d, ls in ((2, (4, 5, 6)), (3, (3, 4, 5))):
        errs = []
        for l in ls:
            lv = (l,) * d
            uh = exact.solve(lv, inputs.ct_rhs(lv))
            X = grid.lex_coords(lv) / float(1 << l)
            errs.append(np.abs(uh - inputs.ct_exact(X)).max())
        for a, b in zip(errs, errs[1:]):
            assert 3.8 < a / b < 4.2, (d, errs)


def test_combination_solution_converges():
    """eq. combi applied to the subgrid solutions of the test problem: the
    combined solution approaches u at second order up to the log factor."""
    d = 2
    pts = inputs.unit_points(10, 300, d)
    ue = inputs.ct_exact(pts)
    errs = []
    for L in (4, 5, 6, 7):
        sols = {lv: exact.solve(lv, inputs.ct_rhs(lv)) for lv, _ in combi.full_layer_set(d, L)}
        errs.append(np.abs(combi.combine(d, L, sols, pts) - ue).max())
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2.5, errs
