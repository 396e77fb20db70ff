"""d-dimensional Hilbert curve and the curve order of the grid points.

Sec. 3.2: the partition is built on the inverse discrete space-filling curve
s_n^{-1}; the paper bases its implementation on Skilling's construction
(J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004) and
uses the isotropic curve at the finest resolution n = max_j l_j (Sec. 3.3).

Readings (the paper fixes none of these):
  * a grid point k is placed at the geometric cell X_j = k_j * 2^{n - l_j};
  * Skilling's axes-to-transpose transform followed by bit interleaving, with
    axis 0 most significant inside each d-bit group, gives the key;
  * the curve starts at the origin cell.
Orientation is a convention: parity unpinned by the paper; bijection, unit-step
continuity and the Hoelder bound of Sec. 3.2 are pinned by tests.

Algorithm 1, step 3: sfc_index orders the grid points by their key.
"""
from __future__ import annotations

import numpy as np

from . import grid


def transpose_form(X: np.ndarray, nbits: int) -> np.ndarray:
    """Skilling's axes -> transpose transform on an (npts, d) array of cell
    coordinates in [0, 2^nbits).  Every point is processed independently; the
    numpy masks run the per-point branches of the published algorithm."""
    X = np.array(X, dtype=np.uint64, copy=True)
    if nbits <= 0:
        return X
    d = X.shape[1]
    top = np.uint64(1) << np.uint64(nbits - 1)
    # undo excess work, from the top bit down to bit 1
    Q = top
    while Q > np.uint64(1):
        low = Q - np.uint64(1)
        for i in range(d):
            hit = (X[:, i] & Q) != 0
            # bit set: invert the low bits of axis 0
            X[hit, 0] ^= low
            # bit clear: exchange the low bits of axis 0 and axis i
            miss = ~hit
            t = (X[miss, 0] ^ X[miss, i]) & low
            X[miss, 0] ^= t
            X[miss, i] ^= t
        Q = Q >> np.uint64(1)
    # Gray encode
    for i in range(1, d):
        X[:, i] ^= X[:, i - 1]
    t = np.zeros(X.shape[0], dtype=np.uint64)
    Q = top
    while Q > np.uint64(1):
        t[(X[:, d - 1] & Q) != 0] ^= Q - np.uint64(1)
        Q = Q >> np.uint64(1)
    for i in range(d):
        X[:, i] ^= t
    return X


def hilbert_key(X: np.ndarray, nbits: int) -> np.ndarray:
    """Hilbert index of each cell: the transpose form's bits read level by level
    from the most significant, axis 0 first within a level."""
    T = transpose_form(X, nbits)
    d = T.shape[1]
    key = np.zeros(T.shape[0], dtype=np.uint64)
    for b in range(nbits - 1, -1, -1):
        for i in range(d):
            key = (key << np.uint64(1)) | ((T[:, i] >> np.uint64(b)) & np.uint64(1))
    return key


def resolution(levels) -> int:
    """n = max_j l_j (Sec. 3.3: finest resolution of an anisotropic grid)."""
    return int(max(levels))


def cells(levels) -> np.ndarray:
    """Geometric cell X_j = k_j * 2^{n - l_j} of every grid point (lex order)."""
    n = resolution(levels)
    K = grid.lex_coords(levels)
    shifts = np.array([n - int(l) for l in levels], dtype=np.int64)
    return (K << shifts[None, :]).astype(np.uint64)


def grid_keys(levels) -> np.ndarray:
    """Hilbert key of every grid point, lexicographic order."""
    levels = tuple(int(l) for l in levels)
    if len(levels) * resolution(levels) > 64:
        raise ValueError("d * max(l) exceeds the 64 bits of a key")
    return hilbert_key(cells(levels), resolution(levels))


def curve_order(levels):
    """Algorithm 1, step 3.  Returns (keys, perm, invperm): perm[pos] is the
    lexicographic id of the point at curve position pos; invperm is its inverse."""
    keys = grid_keys(levels)
    perm = np.argsort(keys, kind="stable").astype(np.int64)
    invperm = np.empty_like(perm)
    invperm[perm] = np.arange(perm.size, dtype=np.int64)
    return keys, perm, invperm
