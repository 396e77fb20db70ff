"""The plain definition of what the solver computes: u = A^{-1} f.

Small grids: dense Cholesky of the assembled A.  Larger grids: a sparse direct
factorization (SuperLU) of A.  Both are library primitives standing for the
exact solution up to rounding.

Any size, including the 4-million-point grids where a sparse direct solve no
longer fits: the sine modes v_m(k) = prod_j sin(pi m_j k_j h_j) are exact
eigenvectors of the Dirichlet finite-difference operator of Sec. 4 with
eigenvalues lambda_m = sum_j 4 c_j / h_j^2 sin^2(pi m_j h_j / 2), and they are
orthogonal, so A^{-1} f = sum_m (v_m^T f / v_m^T v_m) v_m / lambda_m.  The
orthonormal type-I discrete sine transform along every axis is exactly this
change of basis (and its own inverse), so `solve_sine` is a transform, a
pointwise division by lambda_m and the same transform back (a library
primitive, the FFT, for the basis change).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import grid


def solve(levels, f, coeffs=None, dense_limit=5000) -> np.ndarray:
    A = grid.stencil_matrix(levels, coeffs)
    f = np.asarray(f, dtype=np.float64)
    if A.shape[0] <= dense_limit:
        return sla.cho_solve(sla.cho_factor(A.toarray(), lower=True), f)
    return spla.spsolve(A.tocsc(), f)


def sine_eigenvalues(levels, coeffs=None) -> np.ndarray:
    """lambda_m on the full mode grid m_j = 1..2^{l_j}-1 (C order, last axis
    fastest), the closed form of Sec. 4's operator summed over the axes."""
    w = grid.axis_weights(levels, coeffs)
    lam = np.zeros(tuple(grid.axis_sizes(levels)))
    d = len(levels)
    for j, l in enumerate(levels):
        n1 = 1 << int(l)
        m = np.arange(1, n1, dtype=np.float64)
        mu = 4.0 * w[j] * np.sin(np.pi * m / (2.0 * n1)) ** 2
        shape = [1] * d
        shape[j] = n1 - 1
        lam = lam + mu.reshape(shape)
    return lam


def solve_sine(levels, f, coeffs=None) -> np.ndarray:
    """u = A^{-1} f by the sine-mode expansion (exact to rounding, any size)."""
    sizes = tuple(grid.axis_sizes(levels))
    F = np.asarray(f, dtype=np.float64).reshape(sizes)
    Fh = sfft.dstn(F, type=1, norm="ortho")
    Uh = Fh / sine_eigenvalues(levels, coeffs)
    return sfft.idstn(Uh, type=1, norm="ortho").reshape(-1)
