"""The sparse-grid combination technique around the batched solver (Sec. 2).

eq. combi: the solution on the level-L sparse grid is approximated by
    u_c(x) = sum_{i=0}^{d-1} (-1)^i C(d-1, i) sum_{|l|_1 = L + d - 1 - i} u_l(x),
l_j >= 1, where u_l is the finite-difference solution on the anisotropic full grid
of level l and u_l(x) its piecewise multilinear interpolant.  Every subgrid of
layer i is solved with P = P_hat 2^{d-1-i} subdomains (eq. Pchoice), so every
subdomain holds about 2^L / P_hat points whatever the layer.

All subgrids of all d layers are set up together and solved in one batched
CUDA-graph launch (sfcdd_batch_setup_each / sfcdd_batch_solve); the combination is
evaluated at arbitrary points by one kernel (sfcdd_batch_combine).
"""
from __future__ import annotations

from math import comb

import numpy as np
import torch

from . import inputs


def layer_set(d: int, L: int):
    """[(level vector, layer i)] of eq. combi, layer by layer."""
    out = []
    for i in range(d):
        out += [(lv, i) for lv in inputs.combi_levels(d, (L + d - 1 - i,))]
    return out


def coefficient(d: int, i: int) -> int:
    """(-1)^i C(d-1, i), the weight of layer i in eq. combi."""
    return (-1) ** i * comb(d - 1, i)


def subdomain_count(d: int, i: int, P_hat: int, N: int) -> int:
    """eq. Pchoice, P = P_hat 2^{d-1-i}, kept within 2 <= P <= N / 2 for the
    degenerate subgrids (levels 1 on most axes) that have fewer points."""
    return int(max(2, min(P_hat * (1 << (d - 1 - i)), N // 2)))


class Combination:
    """Set up, solve and evaluate the combination technique for one (d, L).

    rhs(levels) gives each subgrid's right-hand side (lexicographic); the
    default is the Poisson test problem of Sec. 4.3."""

    def __init__(self, d: int, L: int, P_hat: int, gamma: float = 0.5, *, precision="fp64",
                 q=0, rhs=inputs.ct_rhs, variant="additive"):
        from .solver import BatchSolver
        self.d, self.L, self.P_hat = int(d), int(L), int(P_hat)
        if self.L < self.d + 1:
            raise ValueError("need L >= d + 1: every subgrid must hold at least 3 points")
        self.subgrids = layer_set(self.d, self.L)
        self.levels = [lv for lv, _ in self.subgrids]
        self.coef = [coefficient(self.d, i) for _, i in self.subgrids]
        self.P = [subdomain_count(self.d, i, self.P_hat, inputs.grid_size(lv))
                  for lv, i in self.subgrids]
        self.batch = BatchSolver(self.levels, self.P, gamma, precision=precision, q=q,
                                 variant=variant)
        f = np.concatenate([rhs(lv) for lv in self.levels])
        self.f = torch.tensor(f, device="cuda")
        self.u = None
        self.stats = None

    def solve(self, rtol=1e-10, maxit=5000):
        self.u, tot, per = self.batch.solve(self.f, rtol=rtol, maxit=maxit)
        self.stats = (tot, per)
        return self.u

    def evaluate(self, points: torch.Tensor) -> torch.Tensor:
        """u_c at points (npts x d, device, in [0, 1]^d)."""
        if self.u is None:
            raise RuntimeError("solve() first")
        return self.batch.combine(self.coef, self.u, points)

    def close(self):
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
