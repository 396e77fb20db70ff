"""The differentiable solve at full size: 255 x 255 x 63 (4,096,575 unknowns),
P = 512, gamma = 1/2, c ~ U[0.5, 2]^3, the paper's q rule (q = 256, N_0 = 131,072).

L = ||u - u_t||^2 is dominated here by ||u_t||^2 (~1.4e6) while dL/dc ~ 1e-3, so
every difference of losses is formed from the solution vectors,
L(+) - L(-) = sum (u+ - u-) (u+ + u- - 2 u_t), which is the same number without
the cancellation of the constant.  Solves to relative residual 1e-12 with FP32
local factors (flexible PCG, FP64 outer iteration; the gradients agree with the
FP64-factor ones to ~1e-14).  Budget: a relative step 1e-3 in c_j gives a
signal of ~2e-3 of |u| against solve noise below kappa(A) 1e-12 ~ 3e-8 of |u|
and an O(h^2) truncation ~1e-6, so the central differences match to 1e-4.
"""
import numpy as np
import pytest
import torch

from oracle import grid
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

NAME = "diff3d_l8x8x6_P512"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def diff_loss(up, um, ut):
    return float(((up - um) * (up + um - 2.0 * ut)).sum())


def test_full_size_gradients():
    from paper_2110_11211_gb300.solver import Solver
    w = inputs.WORKLOADS[NAME]
    levels, P, gamma = w["levels"], w["P"], w["gamma"]
    N = grid.num_unknowns(levels)
    assert N == 4096575
    c = inputs.coefficients(NAME)
    f = torch.tensor(inputs.rhs(NAME, levels), device="cuda")
    ut = torch.tensor(inputs.target(NAME, levels), device="cuda")
    kw = dict(coeffs=c, precision="fp32")
    with Solver(levels, P, gamma, **kw) as s:
        assert s.get_info().q == 256 and s.get_info().N0 == 131072
        u, st = s.solve(f, rtol=1e-12, maxit=3000)
        assert st.true_rel_res <= 2e-12
        gf, gc, _ = s.solve_backward(u, 2.0 * (u - ut), rtol=1e-12, maxit=3000)
        # dL/df along a direction: u(f +- eps v) = u +- eps A^{-1} v exactly
        v = torch.tensor(inputs.uniform(71, N), device="cuda")
        eps = 1e-2
        up, _ = s.solve(f + eps * v, rtol=1e-12, maxit=3000)
        um, _ = s.solve(f - eps * v, rtol=1e-12, maxit=3000)
        fdv = diff_loss(up, um, ut) / (2 * eps)
        assert abs(fdv - float(gf @ v)) <= 1e-7 * abs(fdv)
        # closed form on a sine mode (u_t = 0): L = |v_m|^2 / lam^2,
        # dL/dc_j = -2 |v_m|^2 dlam_j / lam^3, dL/df = 2 v_m / lam^2
        m = (3, 2, 5)
        vm_np = grid.sine_mode(levels, m)
        lam = grid.sine_eigenvalue(levels, m, c)
        vm = torch.tensor(vm_np, device="cuda")
        u2, _ = s.solve(vm, rtol=1e-12, maxit=3000)
        gf2, gc2, _ = s.solve_backward(u2, 2.0 * u2, rtol=1e-12, maxit=3000)
        dl = np.array([4.0 * 4 ** levels[j] * np.sin(np.pi * m[j] / 2 ** (levels[j] + 1)) ** 2
                       for j in range(3)])
        vv = float(vm_np @ vm_np)
        assert np.allclose(gc2, -2.0 * vv / lam ** 3 * dl, rtol=1e-7)
        ref = 2.0 * vm / lam ** 2
        assert float(torch.linalg.norm(gf2 - ref)) <= 1e-7 * float(torch.linalg.norm(ref))
    # central differences in each c_j (fresh setups: the operator changes)
    for j in range(3):
        h = 1e-3 * c[j]
        sol = []
        for sgn in (1.0, -1.0):
            cc = c.copy()
            cc[j] += sgn * h
            with Solver(levels, P, gamma, coeffs=cc, precision="fp32") as s:
                uj, _ = s.solve(f, rtol=1e-12, maxit=3000)
            sol.append(uj)
        fdj = diff_loss(sol[0], sol[1], ut) / (2 * h)
        assert abs(fdj - gc[j]) <= 1e-4 * abs(gc[j]), (j, fdj, gc[j])
