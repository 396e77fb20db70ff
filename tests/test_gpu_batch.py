"""GPU parity of the batched solve of many subgrid problems in one graph launch
(the combination-technique subproblems of Sec. 2) against the oracle.

Every subgrid must reach the same bars as a single solve: true relative
residual <= 2e-10, solution within 1e-8 of the exact solution, and PCG
iteration count within +-1 of the oracle's PCG on that subgrid."""
import numpy as np
import pytest
import torch

from oracle import exact, krylov, schwarz
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def run_batch(levels, P, gamma, precision, seed=71, rtol=1e-10):
    from paper_2110_11211_gb300.solver import BatchSolver
    f = np.concatenate([inputs.uniform(seed + k, inputs.grid_size(lv)) for k, lv in enumerate(levels)])
    with BatchSolver(levels, P, gamma, precision=precision) as b:
        u, tot, per = b.solve(torch.tensor(f, device="cuda"), rtol=rtol)
        offs = b.offsets
    return f, u.cpu().numpy(), tot, per, offs


@pytest.mark.parametrize("d,norms,P,gamma,precision", [
    (2, (6, 7), 4, 0.5, "fp64"), (2, (7, 8), 5, 1.0, "fp64"), (3, (7, 8), 4, 0.5, "fp64"),
    (4, (7, 8), 4, 0.5, "fp64"), (2, (6, 7), 4, 0.5, "fp32"), (3, (7, 8), 4, 0.5, "bf16")])
def test_batched_solves_match_oracle(d, norms, P, gamma, precision):
    levels = [lv for lv in inputs.combi_levels(d, norms) if inputs.grid_size(lv) >= P]
    f, u, tot, per, offs = run_batch(levels, P, gamma, precision)
    assert tot.status == 0 and tot.fail_index == 0
    for k, lv in enumerate(levels):
        fs = f[offs[k]:offs[k + 1]]
        us = u[offs[k]:offs[k + 1]]
        ue = exact.solve(lv, fs)
        assert per[k].true_rel_res <= 2e-10, (lv, per[k].true_rel_res)
        assert np.linalg.norm(us - ue) <= 1e-8 * np.linalg.norm(ue), lv
        if precision == "fp64":
            S = schwarz.Schwarz(lv, P, gamma)
            _, its, _ = krylov.pcg(lambda v: S.A @ v, S.apply, fs, rtol=1e-10)
            assert abs(per[k].iters - its) <= 1, (lv, per[k].iters, its)


def test_batched_matches_single_handle_solves():
    from paper_2110_11211_gb300.solver import Solver
    levels = inputs.combi_levels(3, (7,))
    f, u, tot, per, offs = run_batch(levels, 4, 0.5, "fp64", seed=81)
    for k, lv in enumerate(levels):
        with Solver(lv, 4, 0.5) as s:
            us, st = s.solve(torch.tensor(f[offs[k]:offs[k + 1]], device="cuda"))
        assert abs(st.iters - per[k].iters) <= 1
        ref = us.cpu().numpy()
        assert np.linalg.norm(u[offs[k]:offs[k + 1]] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_combination_set_d4_l12_13_P64():
    """All 385 level vectors of d = 4 with |l|_1 in {12, 13}, P = 64, gamma = 1/2,
    FP32 local factors: every subgrid converges; a sample is checked against
    the exact solution."""
    levels = inputs.combi_levels(4, (12, 13))
    assert len(levels) == 385
    f, u, tot, per, offs = run_batch(levels, 64, 0.5, "fp32", seed=91)
    assert tot.status == 0 and tot.fail_index == 0
    assert max(p.true_rel_res for p in per) <= 2e-10
    for k in range(0, 385, 48):
        lv = levels[k]
        fs = f[offs[k]:offs[k + 1]]
        ue = exact.solve(lv, fs)
        assert np.linalg.norm(u[offs[k]:offs[k + 1]] - ue) <= 1e-8 * np.linalg.norm(ue), lv


def test_more_local_matrices_than_one_grid_dimension():
    """1100 subgrids x 64 subdomains = 70,400 local matrices, beyond the 65,535
    CTAs of one grid dimension: every subgrid still matches its single solve."""
    from paper_2110_11211_gb300.solver import BatchSolver, Solver
    lv = (5, 6)
    n = inputs.grid_size(lv)
    nsub = 1100
    f = torch.tensor(inputs.uniform(97, n * nsub), device="cuda")
    with BatchSolver([lv] * nsub, 64, 0.5, precision="fp32") as b:
        u, tot, per = b.solve(f, rtol=1e-10)
        assert tot.fail_index == 0
        offs = b.offsets
    for s in (0, 517, nsub - 1):
        with Solver(lv, 64, 0.5, precision="fp32") as one:
            us, st = one.solve(f[offs[s]:offs[s + 1]].contiguous(), rtol=1e-10)
        rel = float(torch.linalg.norm(u[offs[s]:offs[s + 1]] - us) / torch.linalg.norm(us))
        assert rel <= 1e-8, (s, rel)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_balanced_batch_equals_single_solves(precision):
    """eq. balSW in the batched solver: every subgrid's solution and iteration
    count equal its single balanced solve (and the oracle's balanced PCG count)."""
    from paper_2110_11211_gb300.solver import BatchSolver, Solver
    levels = [(6, 4), (3, 7), (5, 5), (2, 8), (4, 4)]
    Ps = [8, 6, 16, 4, 5]
    sizes = [inputs.grid_size(lv) for lv in levels]
    f = np.concatenate([inputs.uniform(80 + s, n) for s, n in enumerate(sizes)])
    with BatchSolver(levels, Ps, 0.5, precision=precision, variant="balanced") as b:
        u, tot, per = b.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        offs = b.offsets
        u = u.cpu().numpy()
    assert tot.fail_index == 0
    for s, (lv, P) in enumerate(zip(levels, Ps)):
        fs = f[offs[s]:offs[s + 1]]
        with Solver(lv, P, 0.5, precision=precision, variant="balanced") as one:
            us, st = one.solve(torch.tensor(fs, device="cuda"), rtol=1e-10)
        assert abs(per[s].iters - st.iters) <= 1, (s, per[s].iters, st.iters)
        us = us.cpu().numpy()
        assert np.linalg.norm(u[offs[s]:offs[s + 1]] - us) <= 1e-8 * np.linalg.norm(us)
        if precision == "fp64":
            S = schwarz.Schwarz(lv, P, 0.5)
            _, ko, _ = krylov.pcg(lambda v: S.A @ v, S.apply_balanced, fs, rtol=1e-10)
            assert abs(per[s].iters - ko) <= 1, (s, per[s].iters, ko)


def test_balanced_combination_fewer_iterations_same_solution():
    from paper_2110_11211_gb300.combination import Combination
    pts = torch.tensor(inputs.unit_points(98, 2000, 2), device="cuda")
    out, its = {}, {}
    for variant in ("additive", "balanced"):
        with Combination(2, 11, 8, precision="fp32", variant=variant) as ct:
            ct.solve(rtol=1e-10)
            its[variant] = ct.stats[0].iters
            out[variant] = ct.evaluate(pts)
    assert its["balanced"] < its["additive"], its
    assert float((out["balanced"] - out["additive"]).abs().max()) <= 1e-7 * float(out["additive"].abs().max())


def test_batch_non_finite_rhs_reports_nan():
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import BatchSolver
    levels = [(5, 4), (4, 5)]
    f = inputs.uniform(99, sum(inputs.grid_size(lv) for lv in levels))
    f[3] = float("nan")
    with BatchSolver(levels, 4, 0.5) as b:
        with pytest.raises(SfcddError) as e:
            b.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        assert e.value.code == -6
