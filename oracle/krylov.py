"""Outer iterations around the Schwarz preconditioner.

Sec. 3.3 (after Algorithm 3): the two-level operator is used as the
preconditioner of the conjugate gradient method.  The paper prints no CG
listing; this is the textbook Hestenes-Stiefel preconditioned CG, from x_0 = 0
(or a given x_0), stopped when the recurrence residual satisfies
||r_k||_2 <= rtol ||r_0||_2, or, when a `norm` is given, when
norm(x_k) <= rtol norm(x_0).

Sec. 4 measures convergence on the homogeneous problem (f = 0, solution 0):
from a random x_0 the iterate is the error, and the iteration stops once the
energy norm ||x_k||_A = sqrt(x_k^T A x_k) has dropped by 1e-8 relative to
||x_0||_A.  `energy_norm(apply_A)` gives that stopping quantity.
The flexible variant (Sec. 3.3, for preconditioners that are not exactly
symmetric) replaces beta by the Polak-Ribiere form r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k.

Algorithm 3: damped Richardson x <- x + xi C^{-1}(b - A x), with the optimal
damping xi* = 2 / (lambda_min + lambda_max) of eq. (redrate).

Iteration count = number of updates of x = number of preconditioner applies.
"""
from __future__ import annotations

import numpy as np


def energy_norm(apply_A):
    """x -> ||x||_A = sqrt(x^T A x) (Sec. 4)."""
    return lambda x: float(np.sqrt(max(float(x @ apply_A(x)), 0.0)))


def pcg(apply_A, apply_M, b, rtol=1e-10, maxit=1000, flexible=False, x0=None, norm=None):
    """Returns (x, iterations, history of the stopping quantity relative to its
    value at x_0: the residual norm, or norm(x_k) / norm(x_0) when `norm` is given)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    if norm is None:
        n0 = float(np.linalg.norm(r))
        measure = lambda: float(np.linalg.norm(r)) / n0
    else:
        n0 = norm(x)
        measure = lambda: norm(x) / n0
    if n0 == 0.0:
        return x, 0, [0.0]
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
        rel = measure()
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


def lanczos_extremes(apply_A, apply_M, b, steps):
    """Extreme eigenvalues of C^{-1} A from the Lanczos tridiagonal hidden in
    `steps` CG iterations from x_0 = 0 (the spectrum behind the damping
    xi* = 2 / (lambda_min + lambda_max) of eq. (redrate)).  With alpha_j, beta_j
    the CG step lengths and direction updates:
        T_00 = 1/alpha_0,  T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
        T_{j-1,j} = sqrt(beta_{j-1}) / alpha_{j-1}.
    Returns (lambda_min, lambda_max) of T (Ritz values: inside the spectrum)."""
    b = np.asarray(b, dtype=np.float64)
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for _ in range(steps):
        q = apply_A(p)
        alpha = rz / float(p @ q)
        alphas.append(alpha)
        r = r - alpha * q
        if float(np.linalg.norm(r)) <= 1e-14 * float(np.linalg.norm(b)):
            break
        z = apply_M(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j else 0.0)
        if j:
            T[j - 1, j] = T[j, j - 1] = np.sqrt(betas[j - 1]) / alphas[j - 1]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])
