"""Combination-technique bookkeeping (Sec. 2).

Level vectors of layer i: l in N^d, l_j >= 1, |l|_1 = L + (d - 1) - i, i = 0..d-1;
there are C(L + d - 2 - i, d - 1) of them.  Each gets P = P_hat * 2^{d-1-i}
subdomains (eq. Pchoice).  The total number of subdomains is
    P_hat / (d-1)! * sum_{k=0}^{d-1} 2^{d-1-k} prod_{i=1}^{d-1} (L + d - 1 - k - i)
(Sec. 2, the formula before Table 1).  eq. (combi) combines the subgrid
solutions with the weights (-1)^i C(d-1, i).
"""
from __future__ import annotations

from math import comb, factorial


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
