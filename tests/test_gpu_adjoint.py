"""GPU parity of the differentiable solve u = A(c)^{-1} f with L = ||u - u_t||^2.

Against the oracle's adjoint (plain definition: lambda = A^{-1} 2 (u - u_t),
dL/df = lambda, dL/dc_j = -lambda^T (dA/dc_j) u), against the sine-mode closed
form, and against central finite differences of GPU forward solves.
Tolerances: both sides solve to relative residual 1e-12 (kappa(A) <= ~1e4 here),
so the gradients agree to 1e-7 relative.  Central differences in c carry a
truncation error h^2 L'''(c) / 6 and a rounding floor eps L / (2 h) from the
loss sum itself (L ~ 250 here); h = 1e-4 keeps both below 1e-6 of dL/dc
(h = 1e-5 or 1e-6 would put the rounding floor at 3e-6 or 3e-5 relative).
"""
import numpy as np
import pytest
import torch

from oracle import adjoint, grid
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


CASES = [((4, 5), 6, 0.5), ((3, 3, 3), 5, 1.0), ((4, 3, 2), 8, 0.5)]


def gpu_grad(levels, P, gamma, c, f, ut, precision="fp64"):
    from paper_2110_11211_gb300.solver import Solver
    with Solver(levels, P, gamma, coeffs=c, precision=precision) as s:
        fd = torch.tensor(f, device="cuda")
        u, _ = s.solve(fd, rtol=1e-12)
        gu = 2.0 * (u - torch.tensor(ut, device="cuda"))
        gf, gc, st = s.solve_backward(u, gu, rtol=1e-12)
    return u.cpu().numpy(), gf.cpu().numpy(), np.array(gc)


@pytest.mark.parametrize("levels,P,gamma", CASES)
def test_gradients_match_oracle_adjoint(levels, P, gamma):
    N = grid.num_unknowns(levels)
    c = inputs.uniform(31, len(levels), 0.5, 2.0)
    f = inputs.uniform(32, N)
    ut = inputs.uniform(33, N)
    u, gf, gc = gpu_grad(levels, P, gamma, c, f, ut)
    uo, gfo, gco = adjoint.gradients(levels, f, ut, c)
    assert np.linalg.norm(u - uo) <= 1e-9 * np.linalg.norm(uo)
    assert np.linalg.norm(gf - gfo) <= 1e-7 * np.linalg.norm(gfo)
    assert np.allclose(gc, gco, rtol=1e-7, atol=0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_gradients_mixed_precision(precision):
    levels, P, gamma = (4, 5), 6, 0.5
    N = grid.num_unknowns(levels)
    c = inputs.uniform(41, 2, 0.5, 2.0)
    f = inputs.uniform(42, N)
    ut = inputs.uniform(43, N)
    _, gf, gc = gpu_grad(levels, P, gamma, c, f, ut, precision)
    _, gfo, gco = adjoint.gradients(levels, f, ut, c)
    assert np.linalg.norm(gf - gfo) <= 1e-7 * np.linalg.norm(gfo)
    assert np.allclose(gc, gco, rtol=1e-7, atol=0)


def test_coefficient_gradient_sine_mode_closed_form():
    levels, P, gamma = (5, 4, 3), 8, 0.5
    c = np.array([0.8, 1.7, 1.2])
    m = (3, 2, 5)
    v = grid.sine_mode(levels, m)
    lam = grid.sine_eigenvalue(levels, m, c)
    _, gf, gc = gpu_grad(levels, P, gamma, c, v, np.zeros_like(v))
    dl = np.array([4.0 * 4 ** levels[j] * np.sin(np.pi * m[j] / 2 ** (levels[j] + 1)) ** 2
                   for j in range(3)])
    ref = -2.0 * (v @ v) / lam ** 3 * dl
    assert np.allclose(gc, ref, rtol=1e-7)
    assert np.linalg.norm(gf - 2.0 * v / lam ** 2) <= 1e-7 * np.linalg.norm(2.0 * v / lam ** 2)


def test_central_differences_of_gpu_solves():
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (4, 4, 3), 6, 0.5
    N = grid.num_unknowns(levels)
    c = inputs.uniform(51, 3, 0.5, 2.0)
    f = inputs.uniform(52, N)
    ut = inputs.uniform(53, N)
    fd = torch.tensor(f, device="cuda")
    utd = torch.tensor(ut, device="cuda")

    def loss(cc):
        with Solver(levels, P, gamma, coeffs=cc) as s:
            u, _ = s.solve(fd, rtol=1e-13, maxit=2000)
        return float(((u - utd) ** 2).sum())

    _, gf, gc = gpu_grad(levels, P, gamma, c, f, ut)
    h = 1e-4
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fdj = (loss(c + e) - loss(c - e)) / (2 * h)
        assert abs(fdj - gc[j]) <= 1e-6 * abs(gc[j]), (j, fdj, gc[j])
    # L is quadratic in f: central differences along a direction are exact up to rounding
    vdir = inputs.uniform(54, N)
    with Solver(levels, P, gamma, coeffs=c) as s:
        def lf(ff):
            u, _ = s.solve(torch.tensor(ff, device="cuda"), rtol=1e-13, maxit=2000)
            return float(((u - utd) ** 2).sum())
        fdv = (lf(f + 1e-3 * vdir) - lf(f - 1e-3 * vdir)) / 2e-3
    assert abs(fdv - gf @ vdir) <= 1e-7 * abs(fdv)


def test_autograd_function():
    from paper_2110_11211_gb300.autograd import solve
    levels, P, gamma = (4, 5), 6, 0.5
    N = grid.num_unknowns(levels)
    c0 = inputs.uniform(61, 2, 0.5, 2.0)
    f0 = inputs.uniform(62, N)
    ut = inputs.uniform(63, N)
    f = torch.tensor(f0, device="cuda", requires_grad=True)
    c = torch.tensor(c0, dtype=torch.float64, requires_grad=True)
    u = solve(f, c, levels=levels, P=P, overlap=gamma, rtol=1e-12)
    L = ((u - torch.tensor(ut, device="cuda")) ** 2).sum()
    L.backward()
    _, gfo, gco = adjoint.gradients(levels, f0, ut, c0)
    assert np.linalg.norm(f.grad.cpu().numpy() - gfo) <= 1e-7 * np.linalg.norm(gfo)
    assert np.allclose(c.grad.numpy(), gco, rtol=1e-7)
