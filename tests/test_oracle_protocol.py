"""Pins of the oracle's convergence protocol (Sec. 4): the homogeneous problem
A x = 0 from a random x_0, stopped when the energy norm ||x_k||_A has dropped by
1e-8, for the preconditioned CG method and Algorithm 3.

Every expected value is fixed by the mathematics, not by the oracle itself:
the sine modes of the finite-difference Laplacian are its eigenvectors with
closed-form eigenvalues, so a Richardson step scales mode m by exactly
(1 - xi lambda_m); CG started on a combination of k modes with distinct
eigenvalues terminates in exactly k steps; CG with an exact preconditioner
finishes in one step; CG decreases the energy norm of the error monotonically
and obeys the bound 2 ((sqrt(kappa)-1)/(sqrt(kappa)+1))^k.  The Lanczos
estimate of the extreme eigenvalues is checked against dense eigenvalues.
"""
import math

import numpy as np
import pytest

from oracle import grid, krylov, schwarz
from paper_2110_11211_gb300 import inputs


def _A(levels):
    A = grid.stencil_matrix(levels)
    return A, (lambda v: A @ v)


def test_energy_norm_of_sine_modes():
    """||x||_A^2 = sum_m c_m^2 lambda_m ||v_m||^2 for x = sum_m c_m v_m."""
    levels = (5, 3)
    A, Aop = _A(levels)
    modes = [(1, 1), (4, 2), (17, 7)]
    cs = [0.5, -2.0, 1.25]
    x = sum(c * grid.sine_mode(levels, m) for c, m in zip(cs, modes))
    ref = sum(c * c * grid.sine_eigenvalue(levels, m) * float(grid.sine_mode(levels, m) @
                                                             grid.sine_mode(levels, m))
              for c, m in zip(cs, modes))
    assert abs(krylov.energy_norm(Aop)(x) ** 2 - ref) <= 1e-12 * ref


def test_richardson_on_one_mode_closed_form():
    """x_k = (1 - xi lambda_m)^k x_0: K = ceil(log 1e-8 / log |1 - xi lambda_m|).
    m is the top mode, so every other mode (present at rounding level) contracts
    too and cannot grow into the count."""
    levels = (7,)
    A, Aop = _A(levels)
    m = (2 ** 7 - 1,)
    lam = grid.sine_eigenvalue(levels, m)
    x0 = grid.sine_mode(levels, m)
    en = krylov.energy_norm(Aop)
    for rho in (0.9, -0.6, 0.37):
        xi = (1.0 - rho) / lam
        _, K = krylov.richardson(Aop, lambda v: v.copy(), np.zeros_like(x0), xi, x0=x0,
                                 tol=1e-8, maxit=10000, norm=en)
        expect = math.ceil(math.log(1e-8) / math.log(abs(rho)))
        assert K == expect, (rho, K, expect)


def test_cg_terminates_in_k_steps_on_k_modes():
    levels = (6, 4)
    A, Aop = _A(levels)
    en = krylov.energy_norm(Aop)
    modes = [(1, 1), (3, 2), (9, 5), (40, 13)]
    for k in (1, 2, 3, 4):
        x0 = sum(grid.sine_mode(levels, m) for m in modes[:k])
        x, K, hist = krylov.pcg(Aop, lambda v: v.copy(), np.zeros_like(x0), rtol=1e-8,
                                maxit=100, x0=x0, norm=en)
        assert K == k, (k, K, hist)
        assert hist[-2] > 1e-6


def test_exact_preconditioner_one_step():
    levels = (4, 3)
    A, Aop = _A(levels)
    Ad = A.toarray()
    x0 = inputs.uniform(5, A.shape[0])
    en = krylov.energy_norm(Aop)
    Minv = lambda v: np.linalg.solve(Ad, v)
    _, K, _ = krylov.pcg(Aop, Minv, np.zeros_like(x0), rtol=1e-8, x0=x0, norm=en)
    assert K == 1
    _, K = krylov.richardson(Aop, Minv, np.zeros_like(x0), 1.0, x0=x0, tol=1e-8, norm=en)
    assert K == 1


@pytest.mark.parametrize("levels,P,variant", [((8,), 4, "apply"), ((5, 4), 6, "apply_balanced"),
                                              ((3, 3, 2), 5, "apply")])
def test_pcg_energy_monotone_and_kappa_bound(levels, P, variant):
    S = schwarz.Schwarz(levels, P, 0.5)
    M = getattr(S, variant)
    Aop = lambda v: S.A @ v
    x0 = inputs.uniform(9, S.N)
    _, K, hist = krylov.pcg(Aop, M, np.zeros(S.N), rtol=1e-8, x0=x0,
                            norm=krylov.energy_norm(Aop))
    assert hist[-1] <= 1e-8
    assert all(b <= a * (1 + 1e-10) for a, b in zip(hist, hist[1:]))
    Mm = np.column_stack([M(e) for e in np.eye(S.N)])
    ev = np.linalg.eigvals(Mm @ S.A.toarray()).real
    kappa = ev.max() / ev.min()
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    assert K <= math.ceil(math.log(1e-8 / 2) / math.log(rho))


@pytest.mark.parametrize("levels,P,variant", [((6,), 4, "apply"), ((4, 3), 5, "apply_balanced")])
def test_lanczos_extremes_match_dense(levels, P, variant):
    S = schwarz.Schwarz(levels, P, 0.5)
    M = getattr(S, variant)
    Mm = np.column_stack([M(e) for e in np.eye(S.N)])
    ev = np.linalg.eigvals(Mm @ S.A.toarray()).real
    lo, hi = krylov.lanczos_extremes(lambda v: S.A @ v, M, inputs.uniform(3, S.N), S.N)
    assert abs(lo - ev.min()) <= 1e-6 * ev.min()
    assert abs(hi - ev.max()) <= 1e-8 * ev.max()


def test_balanced_pcg_within_paper_bound_q_2_pow_S_minus_4():
    """Sec. 4.2 (weak scaling, q = 2^{S-4}): the omega-weighted balanced PCG needs
    at most 29 iterations for every S and P; here d = 1, S = 8, P = 16."""
    S = schwarz.Schwarz((12,), 16, 0.5, q=16)
    Aop = lambda v: S.A @ v
    x0 = inputs.uniform(11, S.N)
    _, K, hist = krylov.pcg(Aop, S.apply_balanced, np.zeros(S.N), rtol=1e-8, x0=x0,
                            norm=krylov.energy_norm(Aop))
    assert hist[-1] <= 1e-8
    assert K <= 29
