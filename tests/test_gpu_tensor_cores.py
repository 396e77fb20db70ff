"""The factorizations with their panel and trailing-update tile products on the
tensor cores against the CUDA-core factorizations and the oracle: FP32 local
factors (tcgen05 kind::tf32, hi/lo split, FP32 accumulation), BF16 local factors
(kind::f16 bf16 operands, FP32 accumulation; or the FP32 split rounded to bf16)
and FP64 factors (exact 8-bit digit slices as bf16, exact FP32 accumulation, one
FP64 rounding).

Bars: an FP32 factor is accurate to about kappa(A_i) u_32 whatever unit forms
its tile products (kappa(A_i) up to 1.2e4 on these grids, u_32 = 6e-8, so
kappa u_32 = 7e-4): the FP32 preconditioner apply is within 1e-3 relative of the
FP64 one for both factorizations, and the tensor-core one is within 3x the
CUDA-core one (the split keeps 2^-22 per operand against the 2^-24 of an FP32
rounding, over 64-term sums either way); the solves keep the FP64 outer iteration's 1e-10 true
residual and the exact solution to 1e-8, with iteration counts within +-1 of
the CUDA-core factors'.
"""
import numpy as np
import pytest
import torch

from oracle import exact, grid, schwarz
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


GRIDS = [((6, 6), 8, 0.5), ((9, 5, 3), 64, 1.0), ((10, 5, 3), 128, 1.0), ((5, 4, 3, 3), 32, 0.5),
         ((3, 2, 3, 2), 8, 0.5)]


@pytest.mark.parametrize("levels,P,gamma", GRIDS)
def test_fp32_apply_tensor_cores_vs_fp64(levels, P, gamma):
    from paper_2110_11211_gb300.solver import Solver
    g = torch.tensor(inputs.uniform(71, grid.num_unknowns(levels)), device="cuda")
    with Solver(levels, P, gamma) as s:
        ref = s.apply_precond(g)
    err = {}
    for tc in (1, 0):
        with Solver(levels, P, gamma, precision="fp32", tensor_cores=tc) as s:
            z = s.apply_precond(g)
        err[tc] = float(torch.linalg.norm(z - ref) / torch.linalg.norm(ref))
    print("apply error vs FP64, tensor cores / CUDA cores:", err[1], err[0])
    assert err[0] <= 1e-3 and err[1] <= 1e-3, err
    assert err[1] <= 3.0 * err[0] + 1e-6, err


def test_fp32_apply_tensor_cores_vs_oracle():
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (7, 5), 12, 0.5
    S = schwarz.Schwarz(levels, P, gamma)
    g = inputs.uniform(72, S.N)
    with Solver(levels, P, gamma, precision="fp32", tensor_cores=1) as s:
        z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = S.apply(g)
    assert np.linalg.norm(z - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("levels,P,gamma", GRIDS[:2] + GRIDS[3:])
def test_solve_with_tensor_core_factors(levels, P, gamma, precision):
    """FP32: the TF32-split factor against the CUDA-core one (iterations +-1).
    BF16: the FP32-accurate factor rounded to bf16 (tensor_cores = 2) against the
    CUDA-core one (+-1), and the BF16 factorization (bf16 operands, default),
    whose cheaper local solves may cost a few iterations; every solve keeps the
    FP64 outer iteration's accuracy."""
    from paper_2110_11211_gb300.solver import Solver
    f_np = inputs.uniform(73, grid.num_unknowns(levels))
    f = torch.tensor(f_np, device="cuda")
    ue = exact.solve(levels, f_np)
    its = {}
    modes = (1, 0) if precision == "fp32" else (1, 2, 0)
    for tc in modes:
        with Solver(levels, P, gamma, precision=precision, tensor_cores=tc) as s:
            u, st = s.solve(f, rtol=1e-10, maxit=1000)
        assert st.true_rel_res <= 2e-10
        its[tc] = st.iters
        assert np.linalg.norm(u.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)
    print("iterations by tensor-core mode", precision, levels, its)
    ref = 1 if precision == "fp32" else 2
    assert abs(its[ref] - its[0]) <= 1, its
    if precision == "bf16":
        assert its[1] <= its[2] + max(3, its[2] // 5), its


@pytest.mark.parametrize("levels,P,gamma,tol1,tol2", [((6, 6), 8, 0.5, 5e-2, 1e-2),
                                                      ((5, 4, 3, 3), 32, 0.5, 2e-2, 1e-2),
                                                      ((10, 5, 3), 128, 1.0, 1.0, 3e-2)])
def test_bf16_factorization_apply(levels, P, gamma, tol1, tol2):
    """The BF16 factorization (bf16 operands, FP32 accumulation; tol1) and the
    FP32 factor rounded to bf16 (tol2) against the FP64 apply.  Both are limited
    by bf16's unit roundoff u = 2^-9 times the local condition numbers (2e1 .. 1e4
    on these grids); the bf16 operands of the factorization add that error at
    every panel and trailing update, which at kappa(A_i) ~ 1e4 (the 1023 x 31 x 7
    grid; measured 0.38 against 5e-3 for the rounded FP32 factor) changes the
    apply by tens of percent while the preconditioner stays spectrally close (the
    FP64 outer iteration converges in the same count, see the solve tests)."""
    from paper_2110_11211_gb300.solver import Solver
    g = torch.tensor(inputs.uniform(75, grid.num_unknowns(levels)), device="cuda")
    with Solver(levels, P, gamma) as s:
        ref = s.apply_precond(g)
    err = {}
    for tc in (1, 2):
        with Solver(levels, P, gamma, precision="bf16", tensor_cores=tc) as s:
            z = s.apply_precond(g)
        err[tc] = float(torch.linalg.norm(z - ref) / torch.linalg.norm(ref))
    print("bf16 apply error vs FP64 (bf16 factorization, FP32 factor rounded):", levels, err)
    assert err[1] <= tol1 and err[2] <= tol2, err


def test_batch_tensor_core_factors():
    from paper_2110_11211_gb300.solver import BatchSolver
    levels = inputs.combi_levels(3, (10,))
    f = torch.tensor(inputs.uniform(74, sum(inputs.grid_size(lv) for lv in levels)),
                     device="cuda")
    sol = {}
    for tc in (1, 0):
        with BatchSolver(levels, 16, 0.5, precision="fp32", tensor_cores=tc) as b:
            sol[tc], tot, per = b.solve(f, rtol=1e-10)
        assert tot.fail_index == 0
    assert float(torch.linalg.norm(sol[1] - sol[0]) / torch.linalg.norm(sol[0])) <= 1e-8


def test_invalid_tensor_core_option():
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    with pytest.raises(SfcddError):
        Solver((6, 6), 8, 0.5, precision="fp32", tensor_cores=3)


# FP64 factors from sliced tensor-core products: the same FP64 bar as the
# CUDA-core factorization (apply within 1e-12 of the oracle / of each other)
@pytest.mark.parametrize("levels,P,gamma", GRIDS)
def test_fp64_apply_sliced_products(levels, P, gamma):
    from paper_2110_11211_gb300.solver import Solver
    g = torch.tensor(inputs.uniform(75, grid.num_unknowns(levels)), device="cuda")
    z = {}
    for tc in (1, 0):
        with Solver(levels, P, gamma, precision="fp64", tensor_cores=tc) as s:
            z[tc] = s.apply_precond(g)
    rel = float(torch.linalg.norm(z[1] - z[0]) / torch.linalg.norm(z[0]))
    print("FP64 apply, sliced tensor-core vs CUDA-core factors:", rel)
    assert rel <= 1e-12


def test_fp64_apply_sliced_vs_oracle():
    from paper_2110_11211_gb300.solver import Solver
    for levels, P, gamma in [((7, 5), 12, 0.5), ((4, 4, 3), 10, 1.0)]:
        S = schwarz.Schwarz(levels, P, gamma)
        g = inputs.uniform(76, S.N)
        with Solver(levels, P, gamma, precision="fp64", tensor_cores=1) as s:
            z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
        ref = S.apply(g)
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("levels,P,gamma", GRIDS[:3])
def test_fp64_solve_sliced_products(levels, P, gamma):
    from paper_2110_11211_gb300.solver import Solver
    f_np = inputs.uniform(77, grid.num_unknowns(levels))
    f = torch.tensor(f_np, device="cuda")
    out = {}
    for tc in (1, 0):
        with Solver(levels, P, gamma, precision="fp64", tensor_cores=tc) as s:
            out[tc] = s.solve(f, rtol=1e-10, maxit=1000)
    (u1, st1), (u0, st0) = out[1], out[0]
    assert st1.true_rel_res <= 2e-10 and abs(st1.iters - st0.iters) <= 1
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-9
    ue = exact.solve(levels, f_np)
    assert np.linalg.norm(u1.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)


def test_bf16_factorization_solve_full_size():
    """1023 x 31 x 7, P = 128: the BF16 factorization's larger apply error (see
    above) costs the FP64 outer iteration at most a few percent of its count,
    and the solution keeps the exact solution to 1e-8."""
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (10, 5, 3), 128, 1.0
    f_np = inputs.uniform(inputs.workload_seed("aniso3d_l10x5x3_P128"), grid.num_unknowns(levels))
    ue = exact.solve_sine(levels, f_np)
    f = torch.tensor(f_np, device="cuda")
    its = {}
    for prec, tc in (("fp64", -1), ("bf16", 1), ("bf16", 2)):
        with Solver(levels, P, gamma, precision=prec, tensor_cores=tc) as s:
            u, st = s.solve(f, rtol=1e-10, maxit=1000)
        assert st.true_rel_res <= 2e-10
        assert np.linalg.norm(u.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)
        its[(prec, tc)] = st.iters
    print("iterations fp64 / bf16 factorization / fp32 factor rounded:", its)
    assert its[("bf16", 1)] <= 1.1 * its[("fp64", -1)] + 2, its
