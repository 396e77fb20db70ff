"""Outer iterations around the Schwarz preconditioner.

Sec. 3.3 (after Algorithm 3): the two-level operator is used as the
preconditioner of the conjugate gradient method.  The paper prints no CG
listing; this is the textbook Hestenes-Stiefel preconditioned CG with x_0 = 0,
stopped when the recurrence residual satisfies ||r_k||_2 <= rtol ||b||_2.
The flexible variant (Sec. 3.3, for preconditioners that are not exactly
symmetric) replaces beta by the Polak-Ribiere form r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k.

Algorithm 3: damped Richardson x <- x + xi C^{-1}(b - A x), with the optimal
damping xi* = 2 / (lambda_min + lambda_max) of eq. (redrate).

Iteration count = number of updates of x = number of preconditioner applies.
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, apply_M, b, rtol=1e-10, maxit=1000, flexible=False):
    """Returns (x, iterations, residual-norm history relative to ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, [0.0]
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    hist = [1.0]
    k = 0
    while k < maxit:
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        k += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= rtol:
            break
        z_new = apply_M(r)
        rz_new = float(r @ z_new)
        if flexible:
            beta = float(r @ (z_new - z)) / rz
        else:
            beta = rz_new / rz
        rz = rz_new
        z = z_new
        p = z + beta * p
    return x, k, hist


def richardson(apply_A, apply_M, b, xi, x0=None, tol=1e-8, maxit=10000, norm=None):
    """Algorithm 3.  `norm(x)` is the stopping quantity (the paper tracks the
    energy norm of the error for f = 0); stops when norm(x_k) <= tol * norm(x_0)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if norm is None:
        norm = lambda v: float(np.linalg.norm(b - apply_A(v)))
    n0 = norm(x)
    k = 0
    while k < maxit and norm(x) > tol * n0:
        x = x + xi * apply_M(b - apply_A(x))
        k += 1
    return x, k
