"""The six-dimensional workload at full size: levels (5,4,3,3,2,2), a
31 x 15 x 7 x 7 x 3 x 3 grid of 205,065 unknowns, 13-point stencil, P = 256,
gamma = 1/4, f ~ N(0,1), the paper's q rule (q = 32, N_0 = 8,192) -- the regime
of the dimension study of Sec. 4.2.

Local factors in FP64, FP32 and BF16 (FP32 accumulation in the substitutions);
the outer PCG, the coarse solve, the stencil and the true residual stay in FP64
(flexible beta for the low-precision factors).  Bars:
  - every precision: true relative residual <= 2e-10 at rtol 1e-10 and
    ||u - u*|| <= 1e-8 ||u*|| against the exact solution (sine-mode expansion);
    kappa(A) ~ 1e2 here, so rtol 1e-10 bounds the error far below 1e-8;
  - FP64: the apply against the oracle's apply (eq. addSW, Algorithm 2) element
    by element, |z - z_o| <= 1e-12 max|z_o|, and the PCG iteration count within
    +-1 of the oracle's own PCG, the iterates within 1e-8;
  - FP32 / BF16: the iteration count against FP64's is reported and bounded
    (the penalty of the cheaper local solves).
"""
import numpy as np
import pytest
import torch

from oracle import exact, krylov, schwarz
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

NAME = "aniso6d_l5x4x3x3x2x2_P256"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


@pytest.fixture(scope="module")
def problem():
    w = inputs.WORKLOADS[NAME]
    levels = w["levels"]
    f = inputs.rhs(NAME, levels)
    return levels, w["P"], w["gamma"], f, exact.solve_sine(levels, f)


@pytest.fixture(scope="module")
def gpu_runs(problem):
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma, f, _ = problem
    fd = torch.tensor(f, device="cuda")
    out = {}
    for prec in ("fp64", "fp32", "bf16"):
        with Solver(levels, P, gamma, precision=prec) as s:
            info = s.get_info()
            assert info.q == 32 and info.N0 == 8192
            u, st = s.solve(fd, rtol=1e-10, maxit=1000)
            out[prec] = (u.cpu().numpy(), st)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_solution_against_exact(problem, gpu_runs, prec):
    _, _, _, _, ue = problem
    u, st = gpu_runs[prec]
    assert st.status == 0
    assert st.true_rel_res <= 2e-10, st.true_rel_res
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)


def test_iteration_penalty_of_low_precision_factors(gpu_runs):
    it64 = gpu_runs["fp64"][1].iters
    assert gpu_runs["fp32"][1].iters <= it64 + 2, (gpu_runs["fp32"][1].iters, it64)
    assert gpu_runs["bf16"][1].iters <= 2 * it64 + 10, (gpu_runs["bf16"][1].iters, it64)


def test_fp64_apply_and_pcg_against_oracle(problem, gpu_runs):
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma, f, _ = problem
    S = schwarz.Schwarz(levels, P, gamma)
    g = inputs.normal(77, S.N)
    with Solver(levels, P, gamma) as s:
        z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = S.apply(g)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
    xo, its, _ = krylov.pcg(lambda v: S.A @ v, S.apply, f, rtol=1e-10)
    u, st = gpu_runs["fp64"]
    assert abs(st.iters - its) <= 1, (st.iters, its)
    assert np.linalg.norm(u - xo) <= 1e-8 * np.linalg.norm(xo)
