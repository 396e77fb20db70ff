"""Study definitions of the Sec. 4 iteration experiments (CPU only): the weak-
scaling grids (d = 1: exactly 2^S P - 1 unknowns; d > 1: the largest isotropic
level with d l <= S + log2 P), well-formed study parameters, and the
configurations the partition rejects reported as skipped."""
import math

import pytest

from paper_2110_11211_gb300 import experiments


@pytest.mark.parametrize("S", [6, 8, 10, 12])
def test_weak_levels_keep_two_to_the_s_per_subdomain(S):
    for P in experiments.powers(2, 1024):
        (l,) = experiments.weak_levels(1, S, P)
        assert experiments.grid_size((l,)) == 2 ** S * P - 1
    for d in range(2, 7):
        for P in experiments.powers(2, 1024):
            lv = experiments.weak_levels(d, S, P)
            assert len(lv) == d and len(set(lv)) == 1  # isotropic
            lg = int(math.log2(P))
            # the largest isotropic level with d l <= S + log2 P: at most 2^S unknowns
            # per subdomain (interior points 2^l - 1 per axis)
            assert d * lv[0] <= S + lg < d * (lv[0] + 1)
            assert experiments.grid_size(lv) / P <= 2 ** S


@pytest.mark.parametrize("name", ["E1", "E2", "E3", "E4", "E5", "E6", "E7"])
def test_study_configurations_are_well_formed(name):
    rows = list(experiments.configs(name, 1024))
    assert rows
    for levels, P, gamma, q, variant, weighting in rows:
        assert all(l >= 1 for l in levels) and P >= 2 and gamma > 0 and q >= 1
        assert variant in ("additive", "balanced") and weighting in ("none", "omega")
        if name != "E7":
            assert P & (P - 1) == 0  # powers of two
        else:  # strong scaling: a fixed grid
            assert levels in ((16,), (18,), (20,))


def test_run_one_skips_what_the_partition_rejects():
    # too many coarse blocks, and an overlap that would count a subdomain twice
    row = experiments.run_one((3,), 4, 0.5, 4)
    assert row["skipped"] == "q P > N"
    row = experiments.run_one((8,), 4, 2.0, 1)
    assert row["skipped"] == "2 floor(gamma) + 1 >= P"
