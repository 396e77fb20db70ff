"""The combination technique on the GPU path: per-subgrid subdomain counts
(eq. Pchoice) in one batch, and eq. combi evaluated by sfcdd_batch_combine.

Bars: the combination of given subgrid vectors equals the oracle's
interpolation and combination to rounding, |delta| <= 4 nsub u sum_s |c_s v_s|
(u = 2^-53: the same products summed in another order); the CT solution of the
Sec. 4.3 test problem equals the oracle's (direct subgrid solves) within
1e-6 max|u| (PCG to relative residual 1e-12 on subgrids with kappa < 1e5); every
subgrid of a batch with its own P equals its single solve within 1e-8.
"""
import numpy as np
import pytest
import torch

from oracle import combi, exact
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def oracle_terms(d, L, sols, pts):
    """Per-subgrid weighted interpolants c_s I_s u_s (x_p), shape (nsub, npts)."""
    return np.stack([w * combi.interpolate(lv, sols[lv], pts)
                     for lv, w in combi.full_layer_set(d, L)])


def points_with_nodes_and_edges(d, L, seed):
    pts = inputs.unit_points(seed, 500, d)
    h = 2.0 ** -L
    extra = np.array([[0.5] * d, [h] * d, [1.0 - h] * d, [0.0] * d, [1.0] * d,
                      [0.25 + h / 3] * d])
    return np.vstack([pts, extra])


@pytest.mark.parametrize("d,L,P_hat", [(2, 6, 4), (3, 5, 2), (4, 6, 1)])
def test_combine_matches_oracle_on_given_vectors(d, L, P_hat):
    from paper_2110_11211_gb300.combination import Combination
    with Combination(d, L, P_hat) as ct:
        offs = ct.batch.offsets
        v = inputs.uniform(40 + d, offs[-1])
        sols = {lv: v[offs[s]:offs[s + 1]] for s, lv in enumerate(ct.levels)}
        pts = points_with_nodes_and_edges(d, L, 41)
        out = ct.batch.combine(ct.coef, torch.tensor(v, device="cuda"),
                               torch.tensor(pts, device="cuda")).cpu().numpy()
        out2 = ct.batch.combine(ct.coef, torch.tensor(v, device="cuda"),
                                torch.tensor(pts, device="cuda")).cpu().numpy()
    assert np.array_equal(out, out2)  # fixed summation order
    terms = oracle_terms(d, L, sols, pts)
    ref = terms.sum(axis=0)
    bound = 4 * len(sols) * U * np.abs(terms).sum(axis=0) + 1e-300
    assert np.all(np.abs(out - ref) <= bound), np.max(np.abs(out - ref) / bound)
    assert len(ct.levels) == sum(combi.layer_count(d, L, i) for i in range(d))


@pytest.mark.parametrize("d,L,P_hat", [(2, 7, 4), (3, 5, 2)])
def test_ct_poisson_matches_oracle(d, L, P_hat):
    """Sec. 4.3 test problem: subgrid solves on the GPU + eq. combi against the
    oracle's direct subgrid solves + its own interpolation and combination."""
    from paper_2110_11211_gb300.combination import Combination
    pts = points_with_nodes_and_edges(d, L, 42)
    with Combination(d, L, P_hat) as ct:
        ct.solve(rtol=1e-12)
        tot, per = ct.stats
        assert tot.fail_index == 0
        out = ct.evaluate(torch.tensor(pts, device="cuda")).cpu().numpy()
    sols = {lv: exact.solve(lv, inputs.ct_rhs(lv)) for lv, _ in combi.full_layer_set(d, L)}
    ref = combi.combine(d, L, sols, pts)
    ue = inputs.ct_exact(pts)
    assert np.abs(out - ref).max() <= 1e-6 * np.abs(ue).max()


def test_per_subgrid_subdomain_counts_equal_single_solves():
    from paper_2110_11211_gb300.solver import BatchSolver, Solver
    levels = [(6, 3), (4, 5), (2, 7), (5, 5)]
    Ps = [4, 9, 2, 16]
    f = np.concatenate([inputs.uniform(50 + s, inputs.grid_size(lv))
                        for s, lv in enumerate(levels)])
    with BatchSolver(levels, Ps, 0.5) as b:
        u, tot, per = b.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        offs = b.offsets
        u = u.cpu().numpy()
    for s, (lv, P) in enumerate(zip(levels, Ps)):
        fs = f[offs[s]:offs[s + 1]]
        with Solver(lv, P, 0.5) as one:
            us, st = one.solve(torch.tensor(fs, device="cuda"), rtol=1e-10)
        assert abs(per[s].iters - st.iters) <= 1
        us = us.cpu().numpy()
        assert np.linalg.norm(u[offs[s]:offs[s + 1]] - us) <= 1e-8 * np.linalg.norm(us)
        ue = exact.solve(lv, fs)
        assert np.linalg.norm(us - ue) <= 1e-8 * np.linalg.norm(ue)


@pytest.mark.parametrize("d,Ls,P_hat", [(3, (6, 7, 8, 9), 4), (4, (6, 7, 8, 9), 2)])
def test_ct_solution_converges(d, Ls, P_hat):
    """The combined GPU solution approaches u(x) = ||x|| prod sin(pi x_i) at
    second order up to the logarithmic factor (error ratio per level > 2.5)."""
    from paper_2110_11211_gb300.combination import Combination
    pts = inputs.unit_points(43, 2000, d)
    ue = inputs.ct_exact(pts)
    errs = []
    for L in Ls:
        with Combination(d, L, P_hat, precision="fp32") as ct:
            ct.solve(rtol=1e-10)
            assert ct.stats[0].fail_index == 0
            out = ct.evaluate(torch.tensor(pts, device="cuda")).cpu().numpy()
        errs.append(np.abs(out - ue).max())
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2.5, errs


def test_combine_rejects_bad_arguments():
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.combination import Combination
    with Combination(2, 4, 1) as ct:
        u = torch.zeros(ct.batch.N, dtype=torch.float64, device="cuda")
        pts = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(SfcddError):
            ct.batch.combine([float("nan")] * len(ct.levels), u, pts)
        empty = ct.batch.combine(ct.coef, u, torch.zeros((0, 2), dtype=torch.float64,
                                                         device="cuda"))
        assert empty.numel() == 0
