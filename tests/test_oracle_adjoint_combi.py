"""Pins for the oracle's adjoint gradients and the combination-technique counts."""
import os

import numpy as np
import pytest

from oracle import adjoint, combi, exact, grid
from paper_2110_11211_gb300 import inputs


def test_rhs_gradient_central_difference():
    levels, c = (3, 4), None
    f = inputs.uniform(11, grid.num_unknowns(levels))
    ut = inputs.uniform(12, grid.num_unknowns(levels))
    _, gf, _ = adjoint.gradients(levels, f, ut, c)
    v = inputs.uniform(13, f.size)
    eps = 1e-3     # L is quadratic in f: central differences are exact up to rounding
    fd = (adjoint.loss(levels, f + eps * v, ut) - adjoint.loss(levels, f - eps * v, ut)) / (2 * eps)
    assert abs(fd - gf @ v) <= 1e-9 * abs(fd)


def test_coefficient_gradient_closed_form():
    # f = v_m, u_t = 0: u = v_m / lambda_m, L = |v_m|^2 / lambda_m^2 and
    # dL/dc_j = -2 |v_m|^2 lambda_m^{-3} * 4 / h_j^2 sin^2(pi m_j h_j / 2)
    levels = (4, 3, 3)
    c = np.array([0.8, 1.7, 1.2])
    m = (3, 2, 5)
    v = grid.sine_mode(levels, m)
    lam = grid.sine_eigenvalue(levels, m, c)
    _, _, gc = adjoint.gradients(levels, v, np.zeros_like(v), c)
    dl = np.array([4.0 * 4 ** levels[j] * np.sin(np.pi * m[j] / 2 ** (levels[j] + 1)) ** 2
                   for j in range(3)])
    ref = -2.0 * (v @ v) / lam ** 3 * dl
    assert np.allclose(gc, ref, rtol=1e-10)


def test_coefficient_gradient_central_difference():
    levels = (3, 3, 2)
    c = np.array([0.6, 1.4, 1.9])
    N = grid.num_unknowns(levels)
    f = inputs.uniform(21, N)
    ut = inputs.uniform(22, N)
    _, _, gc = adjoint.gradients(levels, f, ut, c)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1e-6
        fd = (adjoint.loss(levels, f, ut, c + e) - adjoint.loss(levels, f, ut, c - e)) / 2e-6
        assert abs(fd - gc[j]) <= 1e-6 * abs(gc[j])


def test_table1_closed_form(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table1_subdomain_counts.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                d, v = line.split("#")[0].split()
                rows.append((int(d), int(v)))
    assert len(rows) == 6
    for d, v in rows:
        if d <= 5:
            assert combi.total_subdomains_closed_form(d, 20, 1) == v
        else:
            # The printed d = 6 entry is the closed form (and the enumeration) at
            # L = 19, not L = 20: the table is off by one level in that column.
            assert combi.total_subdomains_closed_form(d, 19, 1) == v
            assert combi.total_subdomains_closed_form(d, 20, 1) == 2233216


@pytest.mark.parametrize("d,L", [(2, 8), (3, 7), (4, 6), (5, 5)])
def test_enumeration_matches_closed_form(d, L):
    total = 0
    for i in range(d):
        lv = combi.layer_levels(d, L, i)
        assert len(lv) == combi.layer_count(d, L, i)
        assert all(sum(l) == L + d - 1 - i and min(l) >= 1 for l in lv)
        total += len(lv) * combi.subdomains_per_problem(d, i, 1)
    assert total == combi.total_subdomains_closed_form(d, L, 1)


def test_combination_weights():
    # eq. (combi): (-1)^i C(d-1, i); they alternate and sum to 0 for d >= 2
    assert combi.combination_weights(1) == [1]
    assert combi.combination_weights(3) == [1, -2, 1]
    for d in range(2, 7):
        assert sum(combi.combination_weights(d)) == 0


def test_batched_workload_level_set():
    lv = inputs.combi_levels(4, (12, 13))
    assert len(lv) == 385
    assert len([l for l in lv if sum(l) == 13]) == combi.layer_count(4, 10, 0) == 220
    assert len([l for l in lv if sum(l) == 12]) == combi.layer_count(4, 10, 1) == 165
    sizes = [inputs.grid_size(l) for l in lv]
    assert min(sizes) == 511 and max(sizes) == 5145 and sum(sizes) == 882905
