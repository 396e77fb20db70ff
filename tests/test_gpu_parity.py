"""GPU parity: the CUDA path (through the C-ABI) against the oracle on the same
seeded inputs.

Bars: integer work (keys, curve order, partition, coarse blocks) bit-exact;
FP64 floating point within the bounds derived in the design notes:
  stencil / assembled matrices: same terms summed in another order -> elementwise
  |delta| <= 8 u sum_k |A_ik x_k| (u = 2^-53);
  preconditioner apply (FP64): two triangular solves per subdomain, backward
  stable, relative norm difference <= 1e-12 and every entry within
  1e-12 max_i |z_i| (so one wrong entry of a small subdomain cannot hide);
  solve: ||u - u*|| / ||u*|| <= 1e-8 at relative residual 1e-10 and PCG
  iteration counts within +-1 of the oracle's.
"""
import numpy as np
import pytest
import torch

from oracle import exact, grid, krylov, partition, schwarz, sfc
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def make(levels, P, gamma, **kw):
    from paper_2110_11211_gb300.solver import Solver
    return Solver(levels, P, gamma, **kw)


SMALL = [((5, 4), 6, 0.5), ((3, 3, 3), 5, 1.0), ((7,), 4, 0.25), ((3, 2, 3, 2), 8, 0.5),
         ((2, 2, 2, 2, 2, 2), 9, 0.5), ((6, 6), 8, 0.5), ((4, 5), 7, 0.3), ((2,), 2, 0.5)]


@pytest.mark.parametrize("levels,P,gamma", SMALL + [((10, 5, 3), 128, 1.0),
                                                    ((5, 4, 3, 3, 2, 2), 256, 0.25)])
def test_curve_and_partition_bit_exact(levels, P, gamma):
    kw = dict(variant="coarse_only", q=1) if grid.num_unknowns(levels) > 50000 else {}
    with make(levels, P, gamma, **kw) as s:
        keys, perm = s.curve()
        start, length, omega = s.partition()
    ok, operm, _ = sfc.curve_order(levels)
    assert np.array_equal(keys.cpu().numpy().astype(np.uint64), ok)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
    N = grid.num_unknowns(levels)
    os_, ol = partition.overlap_ranges(N, P, gamma)
    assert np.array_equal(start, os_) and np.array_equal(length, ol)
    assert np.array_equal(omega, partition.omega_weights(N, os_, ol))


def test_curve_at_4m_points():
    # 255 x 255 x 63 grid: keys and curve order at full size (local factors not built)
    levels = (8, 8, 6)
    with make(levels, 512, 0.5, variant="coarse_only", q=1) as s:
        keys, perm = s.curve()
        start, length, _ = s.partition()
    ok, operm, _ = sfc.curve_order(levels)
    assert np.array_equal(keys.cpu().numpy().astype(np.uint64), ok)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
    os_, ol = partition.overlap_ranges(grid.num_unknowns(levels), 512, 0.5)
    assert np.array_equal(start, os_) and np.array_equal(length, ol)


@pytest.mark.parametrize("levels,P,gamma", SMALL)
def test_stencil_matches_assembled_operator(levels, P, gamma):
    N = grid.num_unknowns(levels)
    x = inputs.uniform(7, N)
    c = inputs.uniform(8, len(levels), 0.5, 2.0)
    with make(levels, P, gamma, coeffs=c) as s:
        y = s.apply_operator(torch.tensor(x, device="cuda")).cpu().numpy()
    A = grid.stencil_matrix(levels, c)
    ref = A @ x
    bound = 8 * U * (abs(A) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= bound)


@pytest.mark.parametrize("levels,P,gamma", SMALL)
def test_local_and_coarse_matrices(levels, P, gamma):
    S = schwarz.Schwarz(levels, P, gamma)
    with make(levels, P, gamma) as s:
        A0 = s.coarse_matrix().cpu().numpy()
        locs = [s.local_matrix(i).cpu().numpy() for i in range(min(P, 4))]
    ref0 = S.coarse_matrix()
    assert np.allclose(A0, ref0, rtol=0, atol=64 * U * np.abs(ref0).max())
    for i, Ai in enumerate(locs):
        assert np.array_equal(Ai, S.local_matrix(i))


@pytest.mark.parametrize("levels,P,gamma", SMALL)
@pytest.mark.parametrize("variant", ["additive", "one_level", "coarse_only", "balanced"])
def test_preconditioner_apply_fp64(levels, P, gamma, variant):
    S = schwarz.Schwarz(levels, P, gamma)
    g = inputs.uniform(9, S.N)
    with make(levels, P, gamma, variant=variant) as s:
        z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
    if variant == "additive":
        ref = S.apply(g)
    elif variant == "one_level":
        ref = S.one_level(g)
    elif variant == "balanced":
        ref = S.apply_balanced(g)
    else:
        ref = S.coarse_correction(g)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    # element by element: a wrong entry of one small subdomain cannot hide in the norm
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("levels,P,gamma", [((6, 6), 8, 0.5), ((3, 3, 3), 5, 1.0),
                                            ((3, 2, 3, 2), 8, 0.5), ((7, 4), 16, 0.5)])
def test_solve_balanced(levels, P, gamma):
    """PCG with the balanced operator (eq. balSW) against the oracle's PCG with
    the same operator: iteration counts within +-1, solutions within 1e-8; it
    needs no more iterations than the additive operator (Sec. 4.1)."""
    S = schwarz.Schwarz(levels, P, gamma)
    f = inputs.uniform(15, S.N)
    with make(levels, P, gamma, variant="balanced") as s:
        u, st = s.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        u = u.cpu().numpy()
    with make(levels, P, gamma) as s2:
        _, st_add = s2.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
    ue = exact.solve(levels, f)
    xo, its, _ = krylov.pcg(lambda v: S.A @ v, S.apply_balanced, f, rtol=1e-10)
    assert st.true_rel_res <= 2e-10
    assert abs(st.iters - its) <= 1, (st.iters, its)
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)
    assert np.linalg.norm(u - xo) <= 1e-8 * np.linalg.norm(xo)
    assert st.iters <= st_add.iters


@pytest.mark.parametrize("levels,P,gamma", SMALL)
def test_solve_fp64(levels, P, gamma):
    S = schwarz.Schwarz(levels, P, gamma)
    f = inputs.uniform(10, S.N)
    with make(levels, P, gamma) as s:
        u, st = s.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        u = u.cpu().numpy()
    ue = exact.solve(levels, f)
    xo, its, _ = krylov.pcg(lambda v: S.A @ v, S.apply, f, rtol=1e-10)
    assert st.rel_res <= 1e-10 and st.true_rel_res <= 2e-10
    assert abs(st.iters - its) <= 1, (st.iters, its)
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)
    assert np.linalg.norm(u - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("levels,P,gamma", [((6, 6), 8, 0.5), ((3, 3, 3), 5, 1.0),
                                            ((3, 2, 3, 2), 8, 0.5)])
def test_solve_mixed_precision(levels, P, gamma, precision):
    f = inputs.uniform(11, grid.num_unknowns(levels))
    with make(levels, P, gamma, precision=precision) as s:
        u, st = s.solve(torch.tensor(f, device="cuda"), rtol=1e-10, maxit=500)
        u = u.cpu().numpy()
    ue = exact.solve(levels, f)
    assert st.true_rel_res <= 2e-10
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 5e-2)])
def test_preconditioner_apply_low_precision(precision, tol):
    levels, P, gamma = (6, 6), 8, 0.5
    S = schwarz.Schwarz(levels, P, gamma)
    g = inputs.uniform(12, S.N)
    with make(levels, P, gamma, precision=precision) as s:
        z = s.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = S.apply(g)
    assert np.linalg.norm(z - ref) <= tol * np.linalg.norm(ref)
    assert np.abs(z - ref).max() <= tol * np.abs(ref).max()


def test_deterministic_repeat():
    levels, P, gamma = (6, 6), 8, 0.5
    f = torch.tensor(inputs.uniform(13, grid.num_unknowns(levels)), device="cuda")
    with make(levels, P, gamma) as s:
        u1, st1 = s.solve(f)
        u2, st2 = s.solve(f)
    assert st1.iters == st2.iters
    assert torch.equal(u1, u2)


def test_zero_rhs_and_invalid_arguments():
    from paper_2110_11211_gb300._lib import SfcddError
    with make((4, 4), 4, 0.5) as s:
        u, st = s.solve(torch.zeros(225, dtype=torch.float64, device="cuda"))
        assert st.iters == 0 and torch.count_nonzero(u) == 0
    for args, code in [(((11,) * 6, 4, 0.5), -2), (((4, 4), 3, 1.0), -1), (((4, 4), 4, 0.0), -1),
                       (((2,), 4, 0.5), -1)]:
        with pytest.raises(SfcddError) as e:
            make(*args)
        assert e.value.code == code


def test_full_size_aniso3d_sampled():
    """1023 x 31 x 7 grid, P = 128, gamma = 1 (FP64, as benchmarked): integer
    structure bit-exact, coarse matrix vs oracle, one-level apply of a vector
    supported on one tilde subdomain (three local solves the oracle computes one
    by one), and the solution against a sparse direct solve."""
    levels, P, gamma = (10, 5, 3), 128, 1.0
    S = schwarz.Schwarz(levels, P, gamma, cache_factors=False)
    N = S.N
    with make(levels, P, gamma) as s:
        A0 = s.coarse_matrix().cpu().numpy()
        f = inputs.uniform(inputs.workload_seed("aniso3d_l10x5x3_P128"), N)
        u, st = s.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        u = u.cpu().numpy()
    ref0 = S.coarse_matrix()
    assert np.allclose(A0, ref0, rtol=0, atol=64 * U * np.abs(ref0).max())
    ue = exact.solve(levels, f)
    assert st.true_rel_res <= 2e-10
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)
    # one-level apply restricted to tilde subdomain 37
    t = 37
    offs = partition.tilde_offsets(S.tilde)
    g = np.zeros(N)
    pos = np.arange(offs[t], offs[t] + S.tilde[t])
    g[S.perm[pos]] = inputs.uniform(99, pos.size)
    with make(levels, P, gamma, variant="one_level") as s1:
        z = s1.apply_precond(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = np.zeros(N)
    for i in (t - 1, t, t + 1):
        ids = S.local_ids(i)
        ref[ids] += S.omega[i] * S.local_solve(i, g[ids])
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("levels,P,gamma", [((6, 6), 8, 0.5), ((4, 3, 3), 6, 1.0),
                                            ((3, 2, 3, 2), 8, 0.5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_local_order_does_not_change_the_preconditioner(levels, P, gamma, precision):
    """The numbering inside a subdomain only changes the factor's envelope:
    A_i^{-1} is the same, so applies agree to rounding and solves converge alike."""
    N = grid.num_unknowns(levels)
    g = torch.tensor(inputs.uniform(14, N), device="cuda")
    out = {}
    for order in ("lex", "curve"):
        with make(levels, P, gamma, precision=precision, local_order=order) as s:
            z = s.apply_precond(g).cpu().numpy()
            u, st = s.solve(g, rtol=1e-10)
            out[order] = (z, u.cpu().numpy(), st.iters, s.get_info().factor_bytes)
    tol = 1e-12 if precision == "fp64" else 1e-4
    zl, zc = out["lex"][0], out["curve"][0]
    assert np.linalg.norm(zl - zc) <= tol * np.linalg.norm(zc)
    assert np.linalg.norm(out["lex"][1] - out["curve"][1]) <= 1e-8 * np.linalg.norm(out["curve"][1])
    assert abs(out["lex"][2] - out["curve"][2]) <= 1
    assert out["lex"][3] <= out["curve"][3]
