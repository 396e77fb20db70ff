"""Pins for the oracle's Hilbert map and curve order (Sec. 3.2; Algorithm 1, step 3)."""
import itertools

import numpy as np
import pytest

from oracle import sfc, grid


def full_cells(d, n):
    side = 1 << n
    g = np.array(list(itertools.product(range(side), repeat=d)), dtype=np.uint64)
    return g


@pytest.mark.parametrize("d,n", [(1, 4), (2, 1), (2, 2), (2, 3), (2, 5), (3, 1), (3, 2),
                                 (3, 4), (4, 2), (4, 3), (5, 2), (6, 2)])
def test_bijection_and_unit_steps(d, n):
    X = full_cells(d, n)
    keys = sfc.hilbert_key(X, n)
    # bijection onto [0, 2^{dn})
    assert np.array_equal(np.sort(keys), np.arange(1 << (d * n), dtype=np.uint64))
    # consecutive keys are neighbouring cells (L1 distance exactly one)
    order = np.argsort(keys)
    Xs = X[order].astype(np.int64)
    steps = np.abs(np.diff(Xs, axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    # the curve starts at the origin cell
    assert np.all(Xs[0] == 0)


def test_one_dimensional_curve_is_identity():
    X = np.arange(1 << 7, dtype=np.uint64)[:, None]
    assert np.array_equal(sfc.hilbert_key(X, 7), X[:, 0])


@pytest.mark.parametrize("d,n", [(2, 6), (3, 4), (4, 3)])
def test_hoelder_bound(d, n):
    # Sec. 3.2: |s(x) - s(y)|_2 <= 2 sqrt(d+3) |x - y|^{1/d}.  In cell units the
    # discrete curve satisfies dist(cell(k1), cell(k2)) <= c_s (|k1-k2|+1)^{1/d} + sqrt(d).
    X = full_cells(d, n)
    keys = sfc.hilbert_key(X, n).astype(np.int64)
    rng = np.random.default_rng(7)
    i = rng.integers(0, X.shape[0], 4000)
    j = rng.integers(0, X.shape[0], 4000)
    dist = np.linalg.norm(X[i].astype(np.float64) - X[j].astype(np.float64), axis=1)
    dk = np.abs(keys[i] - keys[j]).astype(np.float64)
    cs = 2.0 * np.sqrt(d + 3)
    assert np.all(dist <= cs * (dk + 1.0) ** (1.0 / d) + np.sqrt(d))


def test_grid_curve_order_is_a_permutation_and_sorted():
    for levels in [(3, 3), (2, 3), (4, 2, 3), (1, 1, 1, 2), (5, 4, 3, 3, 2, 2)]:
        keys, perm, inv = sfc.curve_order(levels)
        N = grid.num_unknowns(levels)
        assert np.array_equal(np.sort(perm), np.arange(N))
        assert np.array_equal(perm[inv], np.arange(N))
        assert np.all(np.diff(keys[perm].astype(np.float64)) > 0)  # distinct keys


def test_anisotropic_cells_use_finest_resolution():
    # Sec. 3.3: the isotropic curve at n = max_j l_j; a level-2 axis inside a
    # level-3 grid sits on every second cell.
    levels = (2, 3)
    C = sfc.cells(levels)
    assert set(C[:, 0].tolist()) == {2, 4, 6}
    assert set(C[:, 1].tolist()) == set(range(1, 8))


def test_key_overflow_rejected():
    with pytest.raises(ValueError):
        sfc.grid_keys((11,) * 6)
