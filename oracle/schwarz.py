"""The two-level overlapping Schwarz operators of Sec. 3.1 and Sec. 3.3, on the
assembled matrix, in lexicographic numbering.

R_i g = g restricted to Omega_i (the points at curve positions start_i..start_i+N_i-1,
cyclic), R_i^T extends by zero; A_i = R_i A R_i^T (Sec. 3.1).  A_i and A_0 are
factored once by Cholesky and applied by forward/backward substitution (Sec. 3.1:
direct solver, factorization in the setup phase).

eq. (csm):    A_0 = R_0 A R_0^T with R_0 from eq. (restr).
eq. (AS2a):   C_(1)^{-1}   = sum_i R_i^T A_i^{-1} R_i.
eq. (w1levprec) / (addSW):
              C_(2),D^{-1} = R_0^T A_0^{-1} R_0 + sum_i omega_i R_i^T A_i^{-1} R_i,
              with D_i = omega_i I (eq. omegai) and D_0 = I.  Algorithm 2 is this
              sum evaluated subdomain by subdomain; the coarse right-hand side of
              its step 3 is R_0 g.
eq. (balan), (balSW):
              F = R_0^T A_0^{-1} R_0, G = I - A F,
              C_(2),D,bal^{-1} = G^T C_(1),D^{-1} G + F.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import grid, partition, sfc


class Schwarz:
    def __init__(self, levels, P, gamma, q=None, coeffs=None, weighting="omega",
                 cache_factors=True):
        self.levels = tuple(int(l) for l in levels)
        self.d = len(self.levels)
        self.N = grid.num_unknowns(self.levels)
        self.P = int(P)
        self.gamma = float(gamma)
        self.coeffs = None if coeffs is None else np.asarray(coeffs, dtype=np.float64)
        self.A = grid.stencil_matrix(self.levels, self.coeffs)
        self.keys, self.perm, self.invperm = sfc.curve_order(self.levels)
        self.tilde = partition.tilde_sizes(self.N, self.P)
        self.start, self.length = partition.overlap_ranges(self.N, self.P, self.gamma)
        self.omega = partition.omega_weights(self.N, self.start, self.length, weighting)
        self.q = partition.paper_q(self.N, self.P) if not q else int(q)
        self.bstart, self.bsize = partition.coarse_blocks(self.N, self.P, self.q)
        self.N0 = self.q * self.P
        self.cache_factors = cache_factors
        self._factors = {}
        self._R0 = None
        self._A0f = None

    # ---- restriction / local problems (Sec. 3.1) ----
    def local_ids(self, i: int) -> np.ndarray:
        """Lexicographic ids of Omega_i in ascending cyclic curve order."""
        pos = partition.positions(self.start[i], self.length[i], self.N)
        return self.perm[pos]

    def local_matrix(self, i: int) -> np.ndarray:
        """A_i = R_i A R_i^T as a dense matrix."""
        ids = self.local_ids(i)
        return self.A[ids][:, ids].toarray()

    def local_factor(self, i: int):
        if i in self._factors:
            return self._factors[i]
        f = sla.cho_factor(self.local_matrix(i), lower=True, check_finite=False)
        if self.cache_factors:
            self._factors[i] = f
        return f

    def local_solve(self, i: int, gi: np.ndarray) -> np.ndarray:
        """d_i = A_i^{-1} g_i (Algorithm 2, step 2)."""
        return sla.cho_solve(self.local_factor(i), gi, check_finite=False)

    # ---- coarse problem (eqs. restr, csm) ----
    @property
    def R0(self) -> sp.csr_matrix:
        if self._R0 is None:
            rows = np.repeat(np.arange(self.N0, dtype=np.int64), self.bsize)
            pos = np.concatenate([np.arange(s, s + n, dtype=np.int64)
                                  for s, n in zip(self.bstart, self.bsize)])
            cols = self.perm[pos]
            self._R0 = sp.csr_matrix((np.ones(rows.size), (rows, cols)),
                                     shape=(self.N0, self.N))
        return self._R0

    def coarse_matrix(self) -> np.ndarray:
        """eq. (csm) by the explicit sparse triple product."""
        R0 = self.R0
        return (R0 @ self.A @ R0.T).toarray()

    def coarse_factor(self):
        if self._A0f is None:
            self._A0f = sla.cho_factor(self.coarse_matrix(), lower=True, check_finite=False)
        return self._A0f

    def coarse_solve(self, g0: np.ndarray) -> np.ndarray:
        """d_0 = A_0^{-1} g_0 (Algorithm 2, step 3)."""
        return sla.cho_solve(self.coarse_factor(), g0, check_finite=False)

    def coarse_correction(self, g: np.ndarray) -> np.ndarray:
        """F g = R_0^T A_0^{-1} R_0 g."""
        return self.R0.T @ self.coarse_solve(self.R0 @ g)

    # ---- preconditioners ----
    def one_level(self, g: np.ndarray, weighted: bool = True) -> np.ndarray:
        """eq. (w1levprec) (weighted) or eq. (AS2a) (weighted=False), summed in i order."""
        h = np.zeros(self.N)
        for i in range(self.P):
            ids = self.local_ids(i)
            di = self.local_solve(i, g[ids])
            h[ids] += (self.omega[i] if weighted else 1.0) * di
        return h

    def apply(self, g: np.ndarray) -> np.ndarray:
        """eq. (addSW) via Algorithm 2: coarse term first, then subdomains in i order."""
        g = np.asarray(g, dtype=np.float64)
        h = self.coarse_correction(g)
        for i in range(self.P):
            ids = self.local_ids(i)
            h[ids] += self.omega[i] * self.local_solve(i, g[ids])
        return h

    def apply_balanced(self, g: np.ndarray) -> np.ndarray:
        """eq. (balSW): G^T C_(1),D^{-1} G g + F g, with G = I - A F and
        G^T = I - F A (A and F are symmetric)."""
        g = np.asarray(g, dtype=np.float64)
        Gg = g - self.A @ self.coarse_correction(g)
        t = self.one_level(Gg)
        return t - self.coarse_correction(self.A @ t) + self.coarse_correction(g)

    # ---- curve-order views used by parity checks ----
    def to_curve(self, v_lex: np.ndarray) -> np.ndarray:
        return np.asarray(v_lex)[self.perm]

    def to_lex(self, v_curve: np.ndarray) -> np.ndarray:
        out = np.empty_like(v_curve)
        out[self.perm] = v_curve
        return out
