"""The convergence protocol of Sec. 4 through the C-ABI (sfcdd_solve_homogeneous):
A x = 0 from a random x_0, stopped when ||x_K||_A <= 1e-8 ||x_0||_A.

Parity with the oracle (oracle.krylov.pcg / richardson with x0 and the energy
norm): after a fixed number of steps the iterates agree to rounding (same
arithmetic in another summation order, relative 1e-10 of ||x_0||), and the
iteration counts at tolerance 1e-8 agree within +-1.
"""
import math

import numpy as np
import pytest
import torch

from oracle import krylov, schwarz
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


# (levels, P, gamma, q, variant, weighting)
CASES = [((8,), 8, 0.5, 16, "balanced", "omega"), ((8,), 8, 0.5, 16, "additive", "none"),
         ((5, 4), 6, 0.5, 0, "additive", "omega"), ((3, 3, 2), 5, 1.0, 2, "balanced", "none"),
         ((2, 2, 2, 2, 2, 2), 9, 0.5, 4, "balanced", "omega"), ((7,), 4, 0.2, 0, "balanced", "omega")]


def oracle_setup(levels, P, gamma, q, variant, weighting):
    S = schwarz.Schwarz(levels, P, gamma, q=q or None, weighting=weighting)
    M = S.apply_balanced if variant == "balanced" else S.apply
    Aop = lambda v: S.A @ v
    return S, M, Aop, krylov.energy_norm(Aop)


def dense_xi(S, M):
    Mm = np.column_stack([M(e) for e in np.eye(S.N)])
    ev = np.linalg.eigvals(Mm @ S.A.toarray()).real
    return 2.0 / (ev.min() + ev.max())


@pytest.mark.parametrize("levels,P,gamma,q,variant,weighting", CASES)
def test_fixed_steps_iterates_match_oracle(levels, P, gamma, q, variant, weighting):
    from paper_2110_11211_gb300.solver import Solver
    S, M, Aop, en = oracle_setup(levels, P, gamma, q, variant, weighting)
    x0 = inputs.uniform(31, S.N)
    xi = dense_xi(S, M)
    with Solver(levels, P, gamma, q=q, variant=variant, weighting=weighting) as s:
        xt = torch.tensor(x0, device="cuda")
        for k in (1, 4):
            u, st = s.solve_homogeneous(xt, "pcg", tol=0.0, maxit=k, check_status=False)
            xo, ko, hist = krylov.pcg(Aop, M, np.zeros(S.N), rtol=0.0, maxit=k, x0=x0, norm=en)
            assert st.iters == ko == k
            assert np.linalg.norm(u.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(x0)
            assert abs(st.true_rel_res - hist[-1]) <= 1e-8 * hist[-1] + 1e-13
            u, st = s.solve_homogeneous(xt, "richardson", xi=xi, tol=0.0, maxit=k,
                                        check_status=False)
            xo, ko = krylov.richardson(Aop, M, np.zeros(S.N), xi, x0=x0, tol=0.0, maxit=k,
                                       norm=en)
            assert st.iters == ko == k
            assert np.linalg.norm(u.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(x0)
            assert abs(st.true_rel_res - en(xo) / en(x0)) <= 1e-8 * en(xo) / en(x0)
        # x0 is not modified
        assert np.array_equal(xt.cpu().numpy(), x0)


@pytest.mark.parametrize("levels,P,gamma,q,variant,weighting", CASES)
def test_counts_match_oracle(levels, P, gamma, q, variant, weighting):
    from paper_2110_11211_gb300.solver import Solver
    S, M, Aop, en = oracle_setup(levels, P, gamma, q, variant, weighting)
    x0 = inputs.uniform(32, S.N)
    xi = dense_xi(S, M)
    _, kp, _ = krylov.pcg(Aop, M, np.zeros(S.N), rtol=1e-8, maxit=5000, x0=x0, norm=en)
    _, kr = krylov.richardson(Aop, M, np.zeros(S.N), xi, x0=x0, tol=1e-8, maxit=100000, norm=en)
    with Solver(levels, P, gamma, q=q, variant=variant, weighting=weighting) as s:
        xt = torch.tensor(x0, device="cuda")
        u, st = s.solve_homogeneous(xt, "pcg", tol=1e-8, maxit=5000)
        assert abs(st.iters - kp) <= 1, (st.iters, kp)
        assert st.true_rel_res <= 1e-8 * (1 + 1e-6)
        assert abs(en(u.cpu().numpy()) / en(x0) - st.true_rel_res) <= 1e-6 * st.true_rel_res
        u, st = s.solve_homogeneous(xt, "richardson", xi=xi, tol=1e-8, maxit=100000)
        assert abs(st.iters - kr) <= 1, (st.iters, kr)
        assert st.true_rel_res <= 1e-8


def test_zero_start_and_invalid_arguments():
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    with Solver((6, 3), 4, 0.5) as s:
        z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        u, st = s.solve_homogeneous(z, "pcg")
        assert st.iters == 0 and float(u.abs().max()) == 0.0
        u, st = s.solve_homogeneous(z, "richardson", xi=0.5)
        assert st.iters == 0 and float(u.abs().max()) == 0.0
        x = torch.ones(s.N, dtype=torch.float64, device="cuda")
        with pytest.raises(SfcddError):
            s.solve_homogeneous(x, "richardson", xi=0.0)
        with pytest.raises(SfcddError):
            s.solve_homogeneous(x, "pcg", tol=-1.0)


def test_estimated_damping_and_paper_ordering_d1():
    """The harness's own path at a moderate size: spectrum estimate -> xi* ->
    Richardson; the balanced operator beats the additive one and PCG beats
    Richardson (Sec. 4.1), and the balanced PCG needs at most 29 steps for
    q = 2^{S-4} (Sec. 4.2)."""
    from paper_2110_11211_gb300 import experiments
    rows = {}
    for variant in ("additive", "balanced"):
        rows[variant] = experiments.run_one(experiments.weak_levels(1, 8, 64), 64, 0.5, 16,
                                            variant, "omega")
    for r in rows.values():
        assert r["pcg"] < r["richardson"]
        assert r["pcg_energy"] <= 1e-8 * (1 + 1e-6) and r["richardson_energy"] <= 1e-8
    assert rows["balanced"]["pcg"] < rows["additive"]["pcg"]
    assert rows["balanced"]["richardson"] < rows["additive"]["richardson"]
    assert rows["balanced"]["pcg"] <= 29


def test_paper_statements_at_scale():
    """The iteration counts the paper states in words (Sec. 4.1, 4.2), at sizes
    on their weak-scaling plateau.  Counts may differ by one from the paper's
    because x_0 is drawn from another generator."""
    from paper_2110_11211_gb300 import experiments as ex
    run = lambda *a: ex.run_one(*a)
    # Sec. 4.1/4.2, d = 1, S = 8, q = 16 = 2^{S-4}, gamma = 1/2
    bal = run(ex.weak_levels(1, 8, 512), 512, 0.5, 16, "balanced", "omega")
    add = run(ex.weak_levels(1, 8, 512), 512, 0.5, 16, "additive", "omega")
    add_none = run(ex.weak_levels(1, 8, 512), 512, 0.5, 16, "additive", "none")
    bal_none = run(ex.weak_levels(1, 8, 512), 512, 0.5, 16, "balanced", "none")
    assert bal["pcg"] <= 29 + 1                        # paper: never more than 29
    assert 120 <= bal["richardson"] <= 170             # paper: levels off near 145
    assert 0.4 <= bal["pcg"] / add["pcg"] <= 0.65      # paper: close to half
    assert add["richardson"] < add_none["richardson"]  # omega scaling helps Richardson
    assert bal["richardson"] == bal_none["richardson"]  # balancing removes the difference
    assert add["richardson"] / bal["richardson"] >= 3.5  # balancing: several times fewer
    # Sec. 4.2, d = 6, isotropic levels 3, S = 8, q = 16: paper: 26 (Richardson), 16 (PCG)
    d6 = run(ex.weak_levels(6, 8, 1024), 1024, 0.5, 16, "balanced", "omega")
    assert d6["levels"] == [3] * 6
    assert 14 <= d6["pcg"] <= 18 and 23 <= d6["richardson"] <= 29
    # Sec. 4.2, q = 16 fixed: the weak-scaling constant grows with S
    s10 = run(ex.weak_levels(1, 10, 256), 256, 0.5, 16, "balanced", "omega")
    assert s10["pcg"] > bal["pcg"] and s10["richardson"] > bal["richardson"]
    # Sec. 4.2, strong scaling L = 16, q = 2^{L-12}: rises with P, peaks, then declines
    its = {P: run((16,), P, 0.5, 16, "balanced", "omega", ("pcg",))["pcg"] for P in (4, 48, 1024)}
    assert its[48] > its[4] and its[48] > its[1024], its
