"""Autotuner of the substitution tile shapes (sfcdd_autotune, sfcdd_batch_autotune).

Every slab shape runs the same arithmetic per row (the same tiles in the same
order, only the rows a CTA covers change), so the preconditioner may differ by
rounding at most (bar: relative 1e-14 in FP64); after tuning, solves equal the
untuned ones to the solve tolerance and the oracle's iteration counts.
Whole-matrix sweeps (slabs_local = -1) form the same products but sum each row
in another order, and are held to the FP64 parity bar against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import exact
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


SHAPES = [(sl, sc) for sl in (1, 2, 4, -1) for sc in (1, 2, 4)]


@pytest.mark.parametrize("precision,variant", [("fp64", "additive"), ("fp64", "balanced"),
                                               ("fp32", "additive"), ("bf16", "additive")])
def test_every_slab_shape_gives_the_same_preconditioner(precision, variant):
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (7, 5, 4), 24, 0.5
    g = torch.tensor(inputs.uniform(61, inputs.grid_size(levels)), device="cuda")
    ref = None
    for sl, sc in SHAPES:
        if precision != "fp64" and sc == 1:
            continue
        with Solver(levels, P, gamma, precision=precision, variant=variant, slabs_local=sl,
                    slabs_coarse=sc) as s:
            z = s.apply_precond(g)
        if ref is None:
            ref = z
        rel = float(torch.linalg.norm(z - ref) / torch.linalg.norm(ref))
        if sl > 0:
            tol = 1e-14 if precision == "fp64" else 1e-6
        else:
            print("whole-matrix vs slab apply", precision, variant, sc, rel)
            tol = 1e-13 if precision == "fp64" else 1e-4
        assert rel <= tol, (sl, sc, rel)


def test_autotune_keeps_the_solution():
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (9, 5, 3), 64, 1.0
    f_np = inputs.uniform(62, inputs.grid_size(levels))
    f = torch.tensor(f_np, device="cuda")
    with Solver(levels, P, gamma) as s:
        u0, st0 = s.solve(f, rtol=1e-10)
        t = s.autotune(reps=3)
        assert t["slabs_local"] in (1, 2, 4, -1) and t["slabs_coarse"] in (1, 2, 4)
        assert t["candidates"] == 12 and t["apply_ms"] > 0
        u1, st1 = s.solve(f, rtol=1e-10)
    assert abs(st1.iters - st0.iters) <= 1
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-9
    ue = exact.solve(levels, f_np)
    assert np.linalg.norm(u1.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)


def test_autotune_low_precision_skips_full_coarse_rows():
    from paper_2110_11211_gb300.solver import Solver
    with Solver((8, 4, 3), 32, 0.5, precision="bf16") as s:
        t = s.autotune(reps=2)
    assert t["candidates"] == 8 and t["slabs_coarse"] in (2, 4)


def test_invalid_slab_options_are_rejected():
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    for kw in (dict(slabs_local=3), dict(slabs_local=-2), dict(slabs_coarse=8),
               dict(precision="fp32", slabs_coarse=1)):
        with pytest.raises(SfcddError):
            Solver((6, 4), 8, 0.5, **kw)


def test_batch_autotune_keeps_the_solutions():
    from paper_2110_11211_gb300.solver import BatchSolver
    levels = inputs.combi_levels(3, (9,))
    f = torch.tensor(inputs.uniform(63, sum(inputs.grid_size(lv) for lv in levels)),
                     device="cuda")
    with BatchSolver(levels, 16, 0.5, precision="fp32") as b:
        u0, tot0, per0 = b.solve(f, rtol=1e-10)
        t = b.autotune(reps=2)
        assert t["candidates"] == 8
        u1, tot1, per1 = b.solve(f, rtol=1e-10)
    assert tot1.fail_index == 0
    assert all(abs(p.iters - q.iters) <= 1 for p, q in zip(per0, per1))
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-9


@pytest.mark.parametrize("variant", ["additive", "balanced", "one_level"])
def test_whole_matrix_apply_vs_oracle(variant):
    from oracle import schwarz
    from paper_2110_11211_gb300.solver import Solver
    for levels, P, gamma in [((7, 5), 12, 0.5), ((4, 4, 3), 10, 1.0), ((3, 2, 3, 2), 8, 0.5)]:
        S = schwarz.Schwarz(levels, P, gamma)
        g = inputs.uniform(64, S.N)
        ref = {"additive": S.apply, "balanced": S.apply_balanced,
               "one_level": S.one_level}[variant](g)
        with Solver(levels, P, gamma, variant=variant, slabs_local=-1) as s:
            z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref), (levels, variant)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max(), (levels, variant)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_whole_matrix_solve(precision):
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (10, 5, 3), 128, 1.0
    f_np = inputs.uniform(65, inputs.grid_size(levels))
    f = torch.tensor(f_np, device="cuda")
    out = {}
    for sl in (1, -1):
        with Solver(levels, P, gamma, precision=precision, slabs_local=sl) as s:
            out[sl] = s.solve(f, rtol=1e-10, maxit=1000)
    (u1, st1), (uw, stw) = out[1], out[-1]
    assert stw.true_rel_res <= 2e-10 and abs(stw.iters - st1.iters) <= 1
    assert float(torch.linalg.norm(uw - u1) / torch.linalg.norm(u1)) <= 1e-8
    ue = exact.solve(levels, f_np)
    assert np.linalg.norm(uw.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)


def test_whole_matrix_batch():
    from paper_2110_11211_gb300.solver import BatchSolver
    levels = inputs.combi_levels(3, (9,))
    f = torch.tensor(inputs.uniform(66, sum(inputs.grid_size(lv) for lv in levels)),
                     device="cuda")
    sol = {}
    for sl in (1, -1):
        for variant in ("additive", "balanced"):
            with BatchSolver(levels, 16, 0.5, variant=variant, slabs_local=sl) as b:
                sol[sl, variant], tot, per = b.solve(f, rtol=1e-10)
            assert tot.fail_index == 0
    for variant in ("additive", "balanced"):
        a, w = sol[1, variant], sol[-1, variant]
        assert float(torch.linalg.norm(w - a) / torch.linalg.norm(a)) <= 1e-8


def test_coarse_block_sizes_vs_oracle():
    """The coarse substitution form L = Lh blockdiag(D_J) with 1-, 2-, 4- and
    8-tile diagonal blocks: the same A_0^{-1}, so the apply meets the FP64 bar."""
    from oracle import schwarz
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (9, 5, 3), 64, 1.0   # N_0 = 4096: 64 coarse tile rows
    S = schwarz.Schwarz(levels, P, gamma)
    g = inputs.uniform(67, S.N)
    ref = S.coarse_correction(g)
    for cb in (1, 2, 4, 8):
        with Solver(levels, P, gamma, variant="coarse_only", coarse_block=cb) as s:
            z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref), cb
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max(), cb
    for cb in (3, 16, -1):
        with pytest.raises(SfcddError):
            Solver((6, 4), 8, 0.5, coarse_block=cb)


def test_whole_matrix_size_limit():
    """Local matrices of about 217 tile rows (1023 x 31 x 7, P = 48, gamma = 1): the
    FP64 matrix vector does not fit beside the ring (at most 189 tile rows), so
    slabs_local = -1 is rejected and the default falls back to row slabs; FP32
    factors (at most 317 tile rows) run whole-matrix items."""
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (10, 5, 3), 48, 1.0
    g = torch.tensor(inputs.uniform(68, inputs.grid_size(levels)), device="cuda")
    with pytest.raises(SfcddError):
        Solver(levels, P, gamma, slabs_local=-1)
    with Solver(levels, P, gamma) as s:
        z_def = s.apply_precond(g)
    with Solver(levels, P, gamma, slabs_local=1) as s:
        z_one = s.apply_precond(g)
    assert float(torch.linalg.norm(z_def - z_one) / torch.linalg.norm(z_one)) == 0.0
    z = {}
    for sl in (-1, 1):
        with Solver(levels, P, gamma, precision="fp32", slabs_local=sl) as s:
            z[sl] = s.apply_precond(g)
    assert float(torch.linalg.norm(z[-1] - z[1]) / torch.linalg.norm(z[1])) <= 1e-4
