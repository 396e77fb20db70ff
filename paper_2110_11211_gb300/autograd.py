"""Differentiable solve u = A(c)^{-1} f.

Forward: sfcdd_setup_ex with the coefficients c, then sfcdd_solve.
Backward: sfcdd_solve_backward runs the adjoint PCG on the same symmetric
preconditioned operator (same factors) and the gradient kernel:
    dL/df = A^{-1} dL/du,  dL/dc_j = -(dL/df)^T (dA/dc_j) u.
"""
from __future__ import annotations

import torch

from .solver import Solver


class SfcddSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, c, levels, P, overlap, rtol, maxit, precision):
        coeffs = None if c is None else [float(v) for v in c.detach().cpu().tolist()]
        solver = Solver(levels, P, overlap, coeffs=coeffs, precision=precision)
        u, _ = solver.solve(f.detach().contiguous().reshape(-1), rtol=rtol, maxit=maxit)
        ctx.solver = solver
        ctx.rtol = rtol
        ctx.maxit = maxit
        ctx.has_c = c is not None
        ctx.c_dtype = None if c is None else c.dtype
        ctx.save_for_backward(u)
        return u.reshape(f.shape)

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        gf, gc, _ = ctx.solver.solve_backward(u, gu.contiguous().reshape(-1), rtol=ctx.rtol,
                                              maxit=ctx.maxit)
        gc_t = torch.tensor(gc, dtype=ctx.c_dtype) if ctx.has_c else None
        ctx.solver.close()
        return gf.reshape(gu.shape), gc_t, None, None, None, None, None, None


def solve(f, c=None, *, levels, P, overlap, rtol=1e-10, maxit=1000, precision="fp64"):
    """u = A(c)^{-1} f with gradients with respect to f and c."""
    return SfcddSolve.apply(f, c, tuple(levels), int(P), float(overlap), float(rtol), int(maxit),
                            precision)
