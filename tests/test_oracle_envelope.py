"""Structure the substitutions rely on, checked on oracle factors (CPU only).

The Cholesky factor L of a symmetric positive definite matrix keeps its row
envelope: L[r, c] = 0 for every c left of the first nonzero of row r of A (no
fill to the left of a row's first nonzero).  Splitting L = Lh D with D the
block diagonal of its 64 x 64 diagonal tiles keeps every zero row of an
off-block tile zero, because Lh_IK = L_IK D_K^{-1}.  So in tile row I the rows
whose envelope starts inside the diagonal tile are exactly zero in all of the
row's off-block tiles, and the transposed tiles have the matching zero
columns.  With the lexicographic numbering inside a curve-ordered subdomain the
bands are narrow, so most rows of the off-block tiles are zero.  These facts
are what lets the substitutions skip those rows exactly.
"""
import numpy as np
import pytest

from oracle import schwarz

TILE = 64


def _lex_local(S, i):
    """A_i with its unknowns in lexicographic order (the GPU path's default
    local numbering; A_i^{-1} does not depend on the order)."""
    ids = np.sort(S.local_ids(i))
    return S.A[ids][:, ids].toarray()


def _first_nonzero(A):
    return np.array([np.flatnonzero(A[r])[0] for r in range(A.shape[0])])


def _unit_form(L):
    """Lh = L D^{-1}, D = blockdiag of the 64 x 64 diagonal tiles of L."""
    n = L.shape[0]
    Lh = np.empty_like(L)
    for K in range(0, n, TILE):
        sl = slice(K, min(n, K + TILE))
        Lh[:, sl] = L[:, sl] @ np.linalg.inv(L[sl, sl])
    return Lh


def _zero_row_counts(A, L, Lh):
    """Checks the exact zeros tile row by tile row; returns the numbers of
    off-block tile rows that are zero and that hold nonzeros."""
    n = A.shape[0]
    nt = (n + TILE - 1) // TILE
    first = _first_nonzero(A)
    zero_rows = nonzero_rows = 0
    for I in range(1, nt):
        r0, r1 = I * TILE, min(n, I * TILE + TILE)
        for r in range(r0, r1):
            left = slice(0, r0)
            if first[r] >= r0:  # envelope starts inside the diagonal tile
                assert np.all(L[r, left] == 0.0), (I, r)
                assert np.all(Lh[r, left] == 0.0), (I, r)
                zero_rows += 1
            else:
                nonzero_rows += 1
        # the bound the setup computes: one past the last row reaching left
        reach = [r - r0 for r in range(r0, r1) if first[r] < r0]
        nzr = (max(reach) + 1) if reach else 0
        assert np.all(Lh[r0 + nzr:r1, :r0] == 0.0)
        # transposed tiles: the zero rows are zero columns of Lh_IK^T
        assert np.all(Lh[r0:r1, :r0].T[:, nzr:] == 0.0)
    return zero_rows, nonzero_rows


@pytest.mark.parametrize("levels,P,gamma,i", [((6, 5, 3), 16, 1.0, 3), ((7, 5), 12, 0.5, 5),
                                              ((4, 4, 3, 3), 10, 1.0, 2)])
def test_off_block_rows_beyond_the_envelope_are_zero(levels, P, gamma, i):
    S = schwarz.Schwarz(levels, P, gamma)
    A = _lex_local(S, i)
    L = np.linalg.cholesky(A)
    zero_rows, nonzero_rows = _zero_row_counts(A, L, _unit_form(L))
    assert zero_rows + nonzero_rows > 0


def test_benchmark_subdomains_have_narrow_bands():
    """On the 1023 x 31 x 7 grid with 128 subdomains (gamma = 1) the curve
    pieces are thin in the coarse axes, so fewer than 40% of the off-block tile
    rows of a local factor hold nonzeros (the rest are skipped exactly)."""
    S = schwarz.Schwarz((10, 5, 3), 128, 1.0)
    for i in (7, 64):
        A = _lex_local(S, i)
        L = np.linalg.cholesky(A)
        zero_rows, nonzero_rows = _zero_row_counts(A, L, _unit_form(L))
        assert nonzero_rows < 0.4 * (zero_rows + nonzero_rows), (i, zero_rows, nonzero_rows)


def test_envelope_is_kept_inside_the_band():
    """No fill left of a row's first nonzero, on a matrix whose envelope is
    irregular (the lexicographic local numbering of a 2-D subdomain)."""
    S = schwarz.Schwarz((7, 6), 12, 1.0)
    A = _lex_local(S, 4)
    L = np.linalg.cholesky(A)
    first = _first_nonzero(A)
    for r in range(A.shape[0]):
        assert np.all(L[r, :first[r]] == 0.0)
        assert L[r, first[r]] != 0.0 or first[r] == r
