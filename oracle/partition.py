"""Disjoint and overlapping partitions of the curve, weights and coarse blocks.

All index sets are sets of curve positions 0..N-1 (0-based here; the paper counts
from 1).

eq. (sloc):     tilde N_i = floor(N/P) + 1 for the first r = N mod P subdomains,
                floor(N/P) for the rest; tilde Omega_i are consecutive.
eq. (enlarge):  Omega_i = tilde Omega_i, the floor(gamma) full neighbours on each
                side, the last ceil(eta tilde N) points of the next one to the left
                and the first floor(eta tilde N) points of the next one to the
                right, eta = gamma - floor(gamma); the enumeration of subdomains
                is cyclic.  Every Omega_i is therefore one cyclic range
                (start_i, N_i).
eq. (Di):       (D_i)_jj = 1 / #{i' : j in Omega_i'}.
eq. (omegai):   omega_i = max_j (D_i)_jj.
Lemma 3.1:      gamma = n/2 gives D_i = omega_i I = I/(2 gamma + 1).
eq. (restr):    tilde Omega_i is cut into q consecutive blocks, the first
                (tilde N_i mod q) of size floor(tilde N_i / q) + 1, the rest
                floor(tilde N_i / q); (R_0)_{(i-1)q+m, j} = 1 iff j in block (i, m).

Reading of gamma: gamma is taken as the rational round(gamma * 2^16) / 2^16, so
ceil(eta tilde N) and floor(eta tilde N) are exact integer operations.  Valid
inputs need 2 floor(gamma) + 1 < P and N_i <= N.
"""
from __future__ import annotations

import numpy as np

GAMMA_DEN = 1 << 16


def tilde_sizes(N: int, P: int) -> np.ndarray:
    """eq. (sloc)."""
    f, r = divmod(N, P)
    return np.array([f + 1] * r + [f] * (P - r), dtype=np.int64)


def tilde_offsets(sizes: np.ndarray) -> np.ndarray:
    """First curve position of each tilde Omega_i (Algorithm 1, step 4)."""
    return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)


def gamma_fixed(gamma: float) -> tuple[int, int]:
    """(floor(gamma), eta * 2^16) under the rational reading of gamma."""
    g = int(round(float(gamma) * GAMMA_DEN))
    return g // GAMMA_DEN, g % GAMMA_DEN


def overlap_ranges(N: int, P: int, gamma: float):
    """eq. (enlarge) as cyclic ranges: returns (start, length) arrays."""
    sizes = tilde_sizes(N, P)
    offs = tilde_offsets(sizes)
    gf, eta = gamma_fixed(gamma)
    if gamma <= 0 or 2 * gf + 1 >= P:
        raise ValueError("need gamma > 0 and 2 floor(gamma) + 1 < P")
    start = np.zeros(P, dtype=np.int64)
    length = np.zeros(P, dtype=np.int64)
    for i in range(P):
        left = (i - gf - 1) % P
        right = (i + gf + 1) % P
        n_left = -((-eta * int(sizes[left])) // GAMMA_DEN)   # ceil(eta * tilde N_left)
        n_right = (eta * int(sizes[right])) // GAMMA_DEN      # floor(eta * tilde N_right)
        core = sum(int(sizes[(i + k) % P]) for k in range(-gf, gf + 1))
        start[i] = (int(offs[left]) + int(sizes[left]) - n_left) % N
        length[i] = n_left + core + n_right
    if np.any(length > N):
        raise ValueError("an overlapping subdomain would exceed the grid")
    return start, length


def overlap_sets_literal(N: int, P: int, gamma: float) -> list[set]:
    """eq. (enlarge) written as set unions, used to check overlap_ranges."""
    sizes = tilde_sizes(N, P)
    offs = tilde_offsets(sizes)
    gf, eta = gamma_fixed(gamma)
    tilde = [set(range(int(offs[i]), int(offs[i] + sizes[i]))) for i in range(P)]
    out = []
    for i in range(P):
        s = set(tilde[i])
        for k in range(1, gf + 1):
            s |= tilde[(i - k) % P] | tilde[(i + k) % P]
        left = (i - gf - 1) % P
        right = (i + gf + 1) % P
        lo = sorted(tilde[left])
        hi = sorted(tilde[right])
        n_left = -((-eta * len(lo)) // GAMMA_DEN)
        n_right = (eta * len(hi)) // GAMMA_DEN
        s |= set(lo[len(lo) - n_left:]) if n_left > 0 else set()
        s |= set(hi[:n_right])
        out.append(s)
    return out


def positions(start: int, length: int, N: int) -> np.ndarray:
    """Curve positions of a cyclic range, in ascending cyclic order from start."""
    return (int(start) + np.arange(int(length), dtype=np.int64)) % N


def coverage_counts(N: int, start, length) -> np.ndarray:
    """#{i : p in Omega_i} for every curve position p (denominator of eq. Di)."""
    cnt = np.zeros(N, dtype=np.int64)
    for s, n in zip(start, length):
        cnt[positions(s, n, N)] += 1
    return cnt


def omega_weights(N: int, start, length, weighting: str = "omega") -> np.ndarray:
    """eq. (omegai) for weighting='omega'; ones for weighting='none'."""
    P = len(start)
    if weighting == "none":
        return np.ones(P)
    cnt = coverage_counts(N, start, length)
    w = np.zeros(P)
    for i in range(P):
        w[i] = np.max(1.0 / cnt[positions(start[i], length[i], N)])
    return w


def paper_q(N: int, P: int) -> int:
    """Coarse dofs per subdomain: the coarse space is kept about four levels
    coarser than the fine one (Sec. 4.1, q = 2^{S-4}; Sec. 4.2, q = 2^{floor(log2(N/P)) - 4}),
    clamped to 1..floor(N/P)."""
    f = N // P
    e = int(np.floor(np.log2(f))) - 4 if f >= 1 else 0
    q = 1 << max(e, 0)
    return int(min(max(q, 1), f))


def coarse_block_sizes(tilde_n: int, q: int) -> np.ndarray:
    """Sizes of the q blocks tilde Omega_{i,m} of one tilde subdomain (Sec. 3.3)."""
    f, r = divmod(int(tilde_n), q)
    return np.array([f + 1] * r + [f] * (q - r), dtype=np.int64)


def coarse_blocks(N: int, P: int, q: int):
    """(start, size) of the N_0 = qP coarse blocks in curve positions, ordered
    by (i, m) as the rows of R_0 in eq. (restr)."""
    sizes = tilde_sizes(N, P)
    if q < 1 or q > int(sizes.min()):
        raise ValueError("need 1 <= q <= floor(N/P)")
    offs = tilde_offsets(sizes)
    bstart, bsize = [], []
    for i in range(P):
        bs = coarse_block_sizes(int(sizes[i]), q)
        o = int(offs[i])
        for m in range(q):
            bstart.append(o)
            bsize.append(int(bs[m]))
            o += int(bs[m])
    return np.array(bstart, dtype=np.int64), np.array(bsize, dtype=np.int64)
