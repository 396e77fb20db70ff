"""Gradients of the quadratic loss L(f, c) = ||u - u_t||_2^2, u = A(c)^{-1} f.

The paper has no adjoint; this is the plain definition used to check the
differentiable solve.  A(c) = sum_j c_j B_j with B_j the axis-j second difference
scaled by 1/h_j^2 (the operator of Sec. 4), so
    lambda  = A^{-1} * 2 (u - u_t)           (A is symmetric)
    dL/df   = lambda
    dL/dc_j = -lambda^T B_j u.
The loss is the plain sum over the interior points (no h^d weight).
`method="sine"` takes both solves by the sine-mode expansion (exact to
rounding at any size); the default uses the dense / sparse direct solve.
"""
from __future__ import annotations

import numpy as np

from . import exact, grid


def _solver(method):
    return exact.solve_sine if method == "sine" else exact.solve


def loss(levels, f, u_t, coeffs=None, method="direct") -> float:
    u = _solver(method)(levels, f, coeffs)
    return float(np.sum((u - u_t) ** 2))


def gradients(levels, f, u_t, coeffs=None, method="direct"):
    """Returns (u, dL/df, dL/dc)."""
    d = len(levels)
    solve = _solver(method)
    u = solve(levels, f, coeffs)
    lam = solve(levels, 2.0 * (u - u_t), coeffs)
    gc = np.array([-float(lam @ (grid.partial_operator(levels, j) @ u)) for j in range(d)])
    return u, lam, gc


def gradients_given(levels, u, lam):
    """dL/dc_j = -lambda^T B_j u for given forward and adjoint fields."""
    d = len(levels)
    return np.array([-float(lam @ (grid.partial_operator(levels, j) @ u)) for j in range(d)])
