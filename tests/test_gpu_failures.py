"""Failure detection without a GPU fault: bounded device waits that give up and
report TIMEOUT, the Cholesky breakdown report, non-finite input, and that the
handle keeps working afterwards.
"""
import numpy as np
import pytest
import torch

from oracle import exact, grid
from paper_2110_11211_gb300 import inputs

pytestmark = pytest.mark.gpu

TIMEOUT, NOT_SPD, NAN = -7, -4, -6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def _solve_ok(s, levels, seed):
    f = inputs.uniform(seed, grid.num_unknowns(levels))
    u, st = s.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
    ue = exact.solve(levels, f)
    assert st.true_rel_res <= 2e-10
    assert np.linalg.norm(u.cpu().numpy() - ue) <= 1e-8 * np.linalg.norm(ue)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bounded_wait_reports_timeout_and_recovers(precision):
    from paper_2110_11211_gb300.solver import Solver
    levels = (7, 5, 3)
    with Solver(levels, 16, 0.5, precision=precision) as s:
        _solve_ok(s, levels, 91)
        rc, site = s.selftest("wait_timeout")
        assert rc == TIMEOUT, rc
        assert site > 0, site  # the wait site that gave up first
        _solve_ok(s, levels, 92)               # same handle, same factors: still correct
        rc, site = s.selftest("wait_timeout")
        assert rc == TIMEOUT


def test_breakdown_reports_not_spd_with_index():
    from paper_2110_11211_gb300.solver import Solver
    levels = (6, 6)
    with Solver(levels, 8, 0.5) as s:
        rc, index = s.selftest("breakdown")
        assert rc == NOT_SPD and index == 4242
        _solve_ok(s, levels, 93)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_rhs_reports_nan(bad):
    from paper_2110_11211_gb300._lib import SfcddError
    from paper_2110_11211_gb300.solver import Solver
    levels = (6, 5)
    f = inputs.uniform(94, grid.num_unknowns(levels))
    f[17] = bad
    with Solver(levels, 8, 0.5) as s:
        with pytest.raises(SfcddError) as e:
            s.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
        assert e.value.code == NAN
        _solve_ok(s, levels, 95)


def test_selftest_rejects_unknown_kind():
    from paper_2110_11211_gb300._lib import lib
    from paper_2110_11211_gb300.solver import Solver
    import ctypes as C
    with Solver((5, 5), 4, 0.5) as s:
        d = C.c_int()
        assert lib().sfcdd_selftest(s._h, 7, C.byref(d)) == -1
