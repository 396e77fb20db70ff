"""The seeded input generators every test and the benchmark share (CPU only).

SplitMix64 is pinned to its published definition (a scalar reference with
Python integers, and the generator's well-known first output for seed 0); the
derived uniform and normal draws to their ranges and moments; the workload
helpers to closed-form counts; the Sec. 4.3 right-hand side to a central
difference Laplacian of the exact solution.
"""
from math import comb

import numpy as np
import pytest

from paper_2110_11211_gb300 import inputs

M64 = (1 << 64) - 1


def splitmix64_scalar(seed, n):
    x, out = seed & M64, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & M64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_first_output_for_seed_zero():
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [0, 1, 0x5FCDD002, (1 << 63) + 12345, M64])
def test_splitmix64_matches_the_scalar_definition(seed):
    got = [int(v) for v in inputs.splitmix64(seed, 1000)]
    assert got == splitmix64_scalar(seed, 1000)


def test_uniform_draws():
    u = inputs.unit_doubles(7, 1 << 20)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))  # 53-bit grid
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    v = inputs.uniform(7, 1000, -3.0, 2.0)
    assert v.min() >= -3.0 and v.max() < 2.0
    assert np.array_equal(inputs.uniform(7, 1000), inputs.uniform(7, 1000))
    assert not np.array_equal(inputs.uniform(7, 1000), inputs.uniform(8, 1000))


def test_normal_draws():
    z = inputs.normal(11, (1 << 20) + 1)  # odd length
    assert z.size == (1 << 20) + 1 and np.all(np.isfinite(z))
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)  # Var(z^4) = 105 - 9


def test_grid_size_and_combination_levels():
    assert inputs.grid_size((10, 5, 3)) == 1023 * 31 * 7
    assert inputs.grid_size((1,)) == 1
    for d in range(1, 6):
        for s in range(d, d + 6):
            lv = inputs.combi_levels(d, (s,))
            assert len(lv) == comb(s - 1, d - 1)  # compositions of s into d parts
            assert all(len(l) == d and sum(l) == s and min(l) >= 1 for l in lv)
            assert lv == sorted(lv) and len(set(lv)) == len(lv)
    # the d = 4 set of the batched workload: |l|_1 in {12, 13}
    assert len(inputs.combi_levels(4, (12, 13))) == comb(11, 3) + comb(12, 3) == 385


def test_workload_seeds_are_distinct():
    seeds = [inputs.workload_seed(w) for w in inputs.WORKLOADS]
    assert len(set(seeds)) == len(seeds)


@pytest.mark.parametrize("levels", [(4, 3), (3, 3, 2), (3, 2, 2, 2)])
def test_ct_rhs_is_minus_the_laplacian_of_ct_exact(levels):
    d = len(levels)
    axes = [np.arange(1, 1 << l, dtype=np.float64) / float(1 << l) for l in levels]
    X = np.stack([g.reshape(-1) for g in np.meshgrid(*axes, indexing="ij")], axis=1)
    h = 1e-4
    lap = np.zeros(X.shape[0])
    u0 = inputs.ct_exact(X)
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        lap += (inputs.ct_exact(X + e) - 2.0 * u0 + inputs.ct_exact(X - e)) / h ** 2
    f = inputs.ct_rhs(levels)
    # central differences: O(h^2) truncation plus about eps |u| / h^2 rounding
    assert np.max(np.abs(f + lap)) <= 1e-5 * max(1.0, np.max(np.abs(f)))
