"""The plain definition of what the solver computes: u = A^{-1} f.

Small grids: dense Cholesky of the assembled A.  Larger grids: a sparse direct
factorization (SuperLU) of A.  Both are library primitives standing for the
exact solution up to rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import grid


def solve(levels, f, coeffs=None, dense_limit=5000) -> np.ndarray:
    A = grid.stencil_matrix(levels, coeffs)
    f = np.asarray(f, dtype=np.float64)
    if A.shape[0] <= dense_limit:
        return sla.cho_solve(sla.cho_factor(A.toarray(), lower=True), f)
    return spla.spsolve(A.tocsc(), f)
