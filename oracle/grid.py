"""Anisotropic full grid and its finite-difference operator.

Sec. 3.3, eq. (dof): interior points k = (k_1..k_d), k_j = 1..2^{l_j}-1, mesh
widths h_j = 2^{-l_j}, N = prod_j (2^{l_j} - 1).

Sec. 4 / Sec. 3.3: the (2d+1)-point finite-difference Laplacian with zero Dirichlet
boundary.  The paper prints no stencil; its remark at the end of Sec. 4.2 (the
level-1 axes of l = (L,1,...,1) contribute a reaction term 8(d-1)) fixes the
scaling to plain 1/h_j^2 coefficients:
    (A u)_k = sum_j c_j / h_j^2 * (2 u_k - u_{k-e_j} - u_{k+e_j}),
with per-axis coefficients c_j (all ones for the Poisson problem).
Lexicographic numbering, last axis fastest (C order).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def num_unknowns(levels) -> int:
    """eq. (dof)."""
    n = 1
    for l in levels:
        n *= (1 << int(l)) - 1
    return n


def axis_sizes(levels):
    return [(1 << int(l)) - 1 for l in levels]


def lex_coords(levels) -> np.ndarray:
    """(N, d) int64 array of interior indices k_j in 1..2^{l_j}-1, row = lex id."""
    sizes = axis_sizes(levels)
    grids = np.meshgrid(*[np.arange(1, s + 1, dtype=np.int64) for s in sizes], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1)


def axis_weights(levels, coeffs=None) -> np.ndarray:
    """c_j / h_j^2 = c_j * 4^{l_j}."""
    d = len(levels)
    c = np.ones(d) if coeffs is None else np.asarray(coeffs, dtype=np.float64)
    return np.array([c[j] * float(4 ** int(levels[j])) for j in range(d)])


def stencil_matrix(levels, coeffs=None) -> sp.csr_matrix:
    """Assembled A in CRS (Algorithm 1, step 7), lexicographic numbering."""
    sizes = axis_sizes(levels)
    d = len(levels)
    N = num_unknowns(levels)
    w = axis_weights(levels, coeffs)
    strides = [1] * d
    for j in range(d - 2, -1, -1):
        strides[j] = strides[j + 1] * sizes[j + 1]
    K = lex_coords(levels)
    ids = np.arange(N, dtype=np.int64)
    rows = [ids]
    cols = [ids]
    vals = [np.full(N, 2.0 * w.sum())]
    for j in range(d):
        for sgn in (-1, 1):
            nb = K[:, j] + sgn
            ok = (nb >= 1) & (nb <= sizes[j])
            rows.append(ids[ok])
            cols.append(ids[ok] + sgn * strides[j])
            vals.append(np.full(int(ok.sum()), -w[j]))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A.tocsr()


def partial_operator(levels, j) -> sp.csr_matrix:
    """dA/dc_j: the axis-j second difference scaled by 1/h_j^2 (used by the adjoint)."""
    d = len(levels)
    e = np.zeros(d)
    e[j] = 1.0
    A = stencil_matrix(levels, coeffs=e)
    return A


def sine_mode(levels, m) -> np.ndarray:
    """v_m(k) = prod_j sin(pi m_j k_j h_j), lexicographic order."""
    K = lex_coords(levels)
    v = np.ones(K.shape[0])
    for j, l in enumerate(levels):
        v *= np.sin(np.pi * m[j] * K[:, j] / float(1 << int(l)))
    return v


def sine_eigenvalue(levels, m, coeffs=None) -> float:
    """Textbook eigenvalue of the Dirichlet FD Laplacian for mode m:
    lambda_m = sum_j 4 c_j / h_j^2 sin^2(pi m_j h_j / 2)."""
    w = axis_weights(levels, coeffs)
    lam = 0.0
    for j, l in enumerate(levels):
        lam += 4.0 * w[j] * np.sin(np.pi * m[j] / float(1 << (int(l) + 1))) ** 2
    return lam
