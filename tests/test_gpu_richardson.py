"""Algorithm 3 (optimally damped preconditioned Richardson iteration) and the
spectrum estimate behind its damping (eq. redrate), through the C-ABI.

The reference spectrum of C^{-1} A comes from dense matrices built with the
oracle (C^{-1} column by column); C^{-1} A is similar to the symmetric
C^{-1/2} A C^{-1/2}, so its eigenvalues are real.  Ritz values of a Lanczos
tridiagonal lie inside the spectrum (Cauchy interlacing), which the estimate
must respect up to rounding.
"""
import numpy as np
import pytest
import torch

from oracle import exact, grid, krylov, schwarz
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


CASES = [((5, 4), 6, 0.5), ((3, 3, 2), 5, 1.0), ((7,), 8, 0.5)]


def dense_spectrum(S, balanced=False):
    apply = S.apply_balanced if balanced else S.apply
    M = np.column_stack([apply(e) for e in np.eye(S.N)])
    ev = np.linalg.eigvals(M @ S.A.toarray()).real
    return float(ev.min()), float(ev.max())


@pytest.mark.parametrize("levels,P,gamma", CASES)
def test_spectrum_estimate_inside_and_close(levels, P, gamma):
    from paper_2110_11211_gb300.solver import Solver
    S = schwarz.Schwarz(levels, P, gamma)
    lo, hi = dense_spectrum(S)
    f = torch.tensor(inputs.uniform(81, S.N), device="cuda")
    with Solver(levels, P, gamma) as s:
        elo, ehi = s.estimate_spectrum(f, steps=S.N)
    assert lo * (1 - 1e-9) <= elo <= ehi <= hi * (1 + 1e-9)
    assert abs(ehi - hi) <= 1e-2 * hi
    assert abs(elo - lo) <= 5e-2 * lo


@pytest.mark.parametrize("levels,P,gamma", CASES)
def test_richardson_matches_oracle(levels, P, gamma):
    """Same damping xi* = 2 / (lambda_min + lambda_max), same stopping rule
    (residual norm): iteration counts within +-1, solution within the tolerance."""
    from paper_2110_11211_gb300.solver import Solver
    S = schwarz.Schwarz(levels, P, gamma)
    lo, hi = dense_spectrum(S)
    xi = 2.0 / (lo + hi)
    f = inputs.uniform(82, S.N)
    rtol = 1e-8
    with Solver(levels, P, gamma) as s:
        u, st = s.richardson(torch.tensor(f, device="cuda"), xi, rtol=rtol, maxit=20000)
        u = u.cpu().numpy()
    xo, ko = krylov.richardson(lambda v: S.A @ v, S.apply, f, xi, tol=rtol, maxit=20000)
    assert abs(st.iters - ko) <= 1, (st.iters, ko)
    assert st.true_rel_res <= rtol
    ue = exact.solve(levels, f)
    assert np.linalg.norm(u - ue) <= 1e-5 * np.linalg.norm(ue)
    # eq. redrate: the contraction 1 - 2 / (1 + kappa) bounds the energy-norm error
    # reduction per step; the residual needs at most a few more steps than that bound
    rho = 1.0 - 2.0 / (1.0 + hi / lo)
    bound = np.log(rtol) / np.log(rho)
    assert st.iters <= 1.5 * bound + 10


def test_estimate_then_iterate_and_balanced_fewer_steps():
    """The practical use (estimate the spectrum, then iterate with the damping
    it gives) converges, and the balanced operator needs fewer Richardson steps
    than the additive one (Sec. 4.1)."""
    from paper_2110_11211_gb300.solver import Solver
    levels, P, gamma = (8,), 16, 0.5
    N = grid.num_unknowns(levels)
    f = torch.tensor(inputs.uniform(83, N), device="cuda")
    its = {}
    for variant in ("additive", "balanced"):
        with Solver(levels, P, gamma, variant=variant) as s:
            lo, hi = s.estimate_spectrum(f, steps=400)
            u, st = s.richardson(f, 2.0 / (lo + hi), rtol=1e-8, maxit=50000)
            its[variant] = st.iters
            assert st.true_rel_res <= 1e-8
    assert its["balanced"] < its["additive"], its
