"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the solver: only the SplitMix64 generator
(S. Vigna's published definition), the derived uniform / normal draws, and the
workload descriptions (grid levels, subdomain count, overlap, precision) of the
problems the solver is exercised on.

SplitMix64: state_k = seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64), then
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31.  A double in [0, 1) is (z >> 11) * 2^-53.  Normal draws use the
Box-Muller transform on consecutive pairs.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs (uint64) for the given seed."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def unit_doubles(seed: int, n: int) -> np.ndarray:
    """n doubles uniformly distributed in [0, 1)."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniformly distributed in [lo, hi)."""
    return lo + (hi - lo) * unit_doubles(seed, n)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on consecutive uniform pairs)."""
    m = (n + 1) // 2
    u = unit_doubles(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]: keeps log finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n]


def grid_size(levels) -> int:
    n = 1
    for l in levels:
        n *= (1 << int(l)) - 1
    return n


# Workloads.  Each names the grid levels l (h_j = 2^-l_j), the subdomain count P,
# the overlap parameter gamma, the right-hand-side distribution and the local
# factor precision.  Seeds: 0x5FCDD000 + index; targets and coefficients use
# seed + 100 and seed + 200.
WORKLOADS = {
    "poisson2d_l6x6_P8": dict(
        index=1, levels=(6, 6), P=8, gamma=0.5, rhs="uniform", precision="fp64",
        coeffs=None),
    "aniso3d_l10x5x3_P128": dict(
        index=2, levels=(10, 5, 3), P=128, gamma=1.0, rhs="uniform", precision="fp64",
        coeffs=None),
    "aniso6d_l5x4x3x3x2x2_P256": dict(
        index=3, levels=(5, 4, 3, 3, 2, 2), P=256, gamma=0.25, rhs="normal",
        precision="fp32", coeffs=None),
    "combi4d_l12-13_P64": dict(
        index=4, levels=None, P=64, gamma=0.5, rhs="uniform", precision="fp32",
        coeffs=None),
    "diff3d_l8x8x6_P512": dict(
        index=5, levels=(8, 8, 6), P=512, gamma=0.5, rhs="uniform", precision="fp64",
        coeffs="uniform_0.5_2"),
}


def workload_seed(name: str) -> int:
    return 0x5FCDD000 + WORKLOADS[name]["index"]


def rhs(name: str, levels=None) -> np.ndarray:
    """Right-hand side f in lexicographic order (last axis fastest)."""
    w = WORKLOADS[name]
    lv = levels if levels is not None else w["levels"]
    n = grid_size(lv)
    seed = workload_seed(name)
    if w["rhs"] == "normal":
        return normal(seed, n)
    return uniform(seed, n, -1.0, 1.0)


def target(name: str, levels=None) -> np.ndarray:
    """Seeded target field u_t for the quadratic loss ||u - u_t||^2."""
    lv = levels if levels is not None else WORKLOADS[name]["levels"]
    return uniform(workload_seed(name) + 100, grid_size(lv), -1.0, 1.0)


def coefficients(name: str) -> np.ndarray | None:
    """Per-axis coefficients c_j (None means all ones)."""
    w = WORKLOADS[name]
    if w["coeffs"] is None:
        return None
    d = len(w["levels"])
    return uniform(workload_seed(name) + 200, d, 0.5, 2.0)


def combi_levels(d: int, norms) -> list[tuple[int, ...]]:
    """All level vectors l in N^d with every l_j >= 1 and |l|_1 in `norms`,
    in lexicographic order (used for the batched combination-method set)."""
    out = []

    def rec(prefix, remaining, slots):
        if slots == 1:
            if remaining >= 1:
                out.append(tuple(prefix + [remaining]))
            return
        for v in range(1, remaining - slots + 2):
            rec(prefix + [v], remaining - v, slots - 1)

    for s in sorted(norms):
        rec([], s, d)
    return out


def unit_points(seed: int, n: int, d: int) -> np.ndarray:
    """n points uniformly distributed in [0, 1)^d, shape (n, d)."""
    return unit_doubles(seed, n * d).reshape(n, d)


def ct_exact(points) -> np.ndarray:
    """The solution of the Poisson test problem of the combination-technique
    study (Sec. 4.3): u(x) = ||x||_2 prod_i sin(pi x_i), zero on the boundary
    of [0, 1]^d.  points: (n, d)."""
    x = np.asarray(points, dtype=np.float64)
    return np.linalg.norm(x, axis=1) * np.prod(np.sin(np.pi * x), axis=1)


def ct_rhs(levels) -> np.ndarray:
    """f = -Laplace(u) of that solution at the interior grid points
    x_j = k_j 2^{-l_j}, lexicographic (last axis fastest).  With r = ||x||_2 and
    s = prod_i sin(pi x_i):  Laplace(u) = s (d-1)/r + 2 (x/r) . grad(s) - d pi^2 r s,
    grad(s)_i = pi cos(pi x_i) prod_{j != i} sin(pi x_j)."""
    levels = [int(l) for l in levels]
    d = len(levels)
    axes = [np.arange(1, 1 << l, dtype=np.float64) / float(1 << l) for l in levels]
    X = np.stack([g.reshape(-1) for g in np.meshgrid(*axes, indexing="ij")], axis=1)
    r = np.linalg.norm(X, axis=1)
    S = np.sin(np.pi * X)
    s = np.prod(S, axis=1)
    grad_dot = np.zeros(X.shape[0])
    for i in range(d):
        others = np.prod(np.delete(S, i, axis=1), axis=1) if d > 1 else np.ones(X.shape[0])
        grad_dot += X[:, i] * np.pi * np.cos(np.pi * X[:, i]) * others
    lap = s * (d - 1) / r + 2.0 * grad_dot / r - d * np.pi ** 2 * r * s
    return -lap
