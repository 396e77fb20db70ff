"""Combination-technique bookkeeping (Sec. 2).

Level vectors of layer i: l in N^d, l_j >= 1, |l|_1 = L + (d - 1) - i, i = 0..d-1;
there are C(L + d - 2 - i, d - 1) of them.  Each gets P = P_hat * 2^{d-1-i}
subdomains (eq. Pchoice).  The total number of subdomains is
    P_hat / (d-1)! * sum_{k=0}^{d-1} 2^{d-1-k} prod_{i=1}^{d-1} (L + d - 1 - k - i)
(Sec. 2, the formula before Table 1).  eq. (combi) combines the subgrid
solutions with the weights (-1)^i C(d-1, i); the combined function is the
weighted sum of the subgrids' piecewise multilinear interpolants, evaluated
here at arbitrary points.
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np


def layer_levels(d: int, L: int, i: int):
    """All level vectors of layer i, by brute-force enumeration."""
    target = L + (d - 1) - i
    out = []

    def rec(prefix, remaining, slots):
        if slots == 1:
            if remaining >= 1:
                out.append(tuple(prefix + [remaining]))
            return
        for v in range(1, remaining - slots + 2):
            rec(prefix + [v], remaining - v, slots - 1)

    rec([], target, d)
    return out


def layer_count(d: int, L: int, i: int) -> int:
    """C(L + d - 2 - i, d - 1)."""
    return comb(L + d - 2 - i, d - 1)


def subdomains_per_problem(d: int, i: int, P_hat: int) -> int:
    """eq. (Pchoice)."""
    return P_hat * (1 << (d - 1 - i))


def total_subdomains_closed_form(d: int, L: int, P_hat: int) -> int:
    """The closed form preceding Table 1."""
    s = 0
    for k in range(d):
        prod = 1
        for i in range(1, d):
            prod *= (L + d - 1 - k - i)
        s += (1 << (d - 1 - k)) * prod
    assert s % factorial(d - 1) == 0
    return P_hat * s // factorial(d - 1)


def combination_weights(d: int):
    """eq. (combi): weight of layer i is (-1)^i C(d-1, i)."""
    return [(-1) ** i * comb(d - 1, i) for i in range(d)]


def full_layer_set(d: int, L: int):
    """(level vector, combination weight) of every subproblem of eq. (combi):
    layers i = 0..d-1, weight (-1)^i C(d-1, i)."""
    w = combination_weights(d)
    return [(lv, w[i]) for i in range(d) for lv in layer_levels(d, L, i)]


def interpolate(levels, values_lex, points):
    """Piecewise multilinear interpolant of a grid function with zero Dirichlet
    data (the nodal basis of Sec. 2's full grids), evaluated at points (n, d) in
    [0, 1]^d.  Node k_j of axis j sits at k_j 2^{-l_j}, k_j = 0..2^{l_j}; the
    boundary nodes k_j = 0 and k_j = 2^{l_j} carry 0, the interior ones the
    lexicographic values (last axis fastest)."""
    levels = [int(l) for l in levels]
    d = len(levels)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, d)
    sizes = [(1 << l) - 1 for l in levels]
    U = np.zeros([s + 2 for s in sizes])
    U[tuple(slice(1, s + 1) for s in sizes)] = np.asarray(values_lex).reshape(sizes)
    out = np.zeros(pts.shape[0])
    for p in range(pts.shape[0]):
        base, frac = [], []
        for j in range(d):
            t = pts[p, j] * (1 << levels[j])
            k = min(int(np.floor(t)), (1 << levels[j]) - 1)
            base.append(k)
            frac.append(t - k)
        acc = 0.0
        for corner in range(1 << d):
            wgt = 1.0
            idx = []
            for j in range(d):
                bit = (corner >> j) & 1
                wgt *= frac[j] if bit else 1.0 - frac[j]
                idx.append(base[j] + bit)
            acc += wgt * U[tuple(idx)]
        out[p] = acc
    return out


def combine(d: int, L: int, solutions, points):
    """eq. (combi): sum over the full layer set of weight x interpolant of the
    subproblem's solution.  solutions: dict level vector -> lexicographic values."""
    out = np.zeros(np.asarray(points).reshape(-1, d).shape[0])
    for lv, w in full_layer_set(d, L):
        out += w * interpolate(lv, solutions[lv], points)
    return out
