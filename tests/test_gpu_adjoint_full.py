"""The differentiable solve at full size: 255 x 255 x 63 (4,096,575 unknowns),
P = 512, gamma = 1/2, c ~ U[0.5, 2]^3, the paper's q rule (q = 256, N_0 = 131,072),
FP64 local factors, forward and adjoint solves to relative residual 1e-12.

Oracle: u and lambda = A^{-1} 2 (u - u_t) by the sine-mode expansion (exact to
rounding at this size), dL/df = lambda, dL/dc_j = -lambda^T B_j u.  kappa(A) is
about 2e4, so a relative residual of 1e-12 bounds the solution error by 2e-8;
the gradients are checked at 1e-6 relative:
  - against the oracle's adjoint gradients;
  - against central differences with step 1e-6 c_j of the exact loss (oracle
    solves; truncation ~1e-12, rounding ~1e-9 relative);
  - against central differences of GPU solves, Richardson-extrapolated from the
    steps h = 1e-3 c_j and h/2, which cancels the O(h^2) term: (4 D(h/2) - D(h)) / 3.
L = ||u - u_t||^2 is dominated here by ||u_t||^2 (~1.4e6) while dL/dc ~ 1e-3, so
every difference of losses is formed from the solution vectors,
L(+) - L(-) = sum (u+ - u-) (u+ + u- - 2 u_t), the same number without the
cancellation of the constant.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint, exact, grid
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

NAME = "diff3d_l8x8x6_P512"
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def diff_loss(up, um, ut):
    return float(((up - um) * (up + um - 2.0 * ut)).sum())


@pytest.fixture(scope="module")
def problem():
    w = inputs.WORKLOADS[NAME]
    levels, P, gamma = w["levels"], w["P"], w["gamma"]
    assert grid.num_unknowns(levels) == 4096575
    c = inputs.coefficients(NAME)
    f = inputs.rhs(NAME, levels)
    ut = inputs.target(NAME, levels)
    return levels, P, gamma, c, f, ut


@pytest.fixture(scope="module")
def gpu_gradients(problem):
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma, c, f, ut = problem
    fd = torch.tensor(f, device="cuda")
    utd = torch.tensor(ut, device="cuda")
    with Solver(levels, P, gamma, coeffs=c) as s:
        assert s.get_info().q == 256 and s.get_info().N0 == 131072
        u, st = s.solve(fd, rtol=RTOL, maxit=3000)
        assert st.true_rel_res <= 2 * RTOL
        gf, gc, _ = s.solve_backward(u, 2.0 * (u - utd), rtol=RTOL, maxit=3000)
        # dL/df along a direction: u(f +- eps v) = u +- eps A^{-1} v exactly
        v = torch.tensor(inputs.uniform(71, f.size), device="cuda")
        eps = 1e-2
        up, _ = s.solve(fd + eps * v, rtol=RTOL, maxit=3000)
        um, _ = s.solve(fd - eps * v, rtol=RTOL, maxit=3000)
        fdv = diff_loss(up, um, utd) / (2 * eps)
        gfv = float(gf @ v)
    return u.cpu().numpy(), gf.cpu().numpy(), np.array(gc), fdv, gfv


def test_gradients_against_oracle_adjoint(problem, gpu_gradients):
    levels, P, gamma, c, f, ut = problem
    u, gf, gc, _, _ = gpu_gradients
    uo, gfo, gco = adjoint.gradients(levels, f, ut, c, method="sine")
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)
    assert np.linalg.norm(gf - gfo) <= 1e-6 * np.linalg.norm(gfo)
    assert np.allclose(gc, gco, rtol=1e-6, atol=0), (gc, gco)


def test_rhs_gradient_along_a_direction(gpu_gradients):
    _, _, _, fdv, gfv = gpu_gradients
    assert abs(fdv - gfv) <= 1e-7 * abs(fdv)


def test_coefficient_gradients_against_exact_central_differences(problem, gpu_gradients):
    """Step 1e-6 c_j on the exact loss (oracle solves)."""
    levels, P, gamma, c, f, ut = problem
    gc = gpu_gradients[2]
    for j in range(3):
        h = 1e-6 * c[j]
        cp, cm = c.copy(), c.copy()
        cp[j] += h
        cm[j] -= h
        up = exact.solve_sine(levels, f, cp)
        um = exact.solve_sine(levels, f, cm)
        fdj = diff_loss(up, um, ut) / (2 * h)
        assert abs(fdj - gc[j]) <= 1e-6 * abs(gc[j]), (j, fdj, gc[j])


def test_coefficient_gradients_against_gpu_central_differences(problem, gpu_gradients):
    """Central differences of GPU solves (fresh setups: the operator changes),
    extrapolated from h and h / 2."""
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma, c, f, ut = problem
    gc = gpu_gradients[2]
    fd = torch.tensor(f, device="cuda")
    utd = torch.tensor(ut, device="cuda")

    def central(j, h):
        sol = []
        for sgn in (1.0, -1.0):
            cc = c.copy()
            cc[j] += sgn * h
            with Solver(levels, P, gamma, coeffs=cc) as s:
                uj, st = s.solve(fd, rtol=RTOL, maxit=3000)
                assert st.true_rel_res <= 2 * RTOL
            sol.append(uj)
        return diff_loss(sol[0], sol[1], utd) / (2 * h)

    for j in range(3):
        h = 1e-3 * c[j]
        d1, d2 = central(j, h), central(j, h / 2)
        ext = (4.0 * d2 - d1) / 3.0
        assert abs(ext - gc[j]) <= 1e-6 * abs(gc[j]), (j, d1, d2, ext, gc[j])


def test_sine_mode_closed_form(problem):
    """f = v_m, u_t = 0: L = |v_m|^2 / lam^2, dL/dc_j = -2 |v_m|^2 dlam_j / lam^3,
    dL/df = 2 v_m / lam^2."""
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma, c, _, _ = problem
    m = (3, 2, 5)
    vm_np = grid.sine_mode(levels, m)
    lam = grid.sine_eigenvalue(levels, m, c)
    vm = torch.tensor(vm_np, device="cuda")
    with Solver(levels, P, gamma, coeffs=c) as s:
        u2, _ = s.solve(vm, rtol=RTOL, maxit=3000)
        gf2, gc2, _ = s.solve_backward(u2, 2.0 * u2, rtol=RTOL, maxit=3000)
    dl = np.array([4.0 * 4 ** levels[j] * np.sin(np.pi * m[j] / 2 ** (levels[j] + 1)) ** 2
                   for j in range(3)])
    vv = float(vm_np @ vm_np)
    assert np.allclose(gc2, -2.0 * vv / lam ** 3 * dl, rtol=1e-7)
    ref = 2.0 * vm / lam ** 2
    assert float(torch.linalg.norm(gf2 - ref)) <= 1e-7 * float(torch.linalg.norm(ref))
