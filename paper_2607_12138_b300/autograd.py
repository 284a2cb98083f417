"""Differentiable density-weighted mass solve x = M(rho)^{-1} b, rho = exp(z).

M(rho) = sum_K rho_K P_K^T M_K^1 P_K (H1; the weight enters the pullback of
Eq. piola_mass_pullbacks like det J).  Forward: the library sets rho = exp(z) on the device
and runs one BRAS-PCG solve.  Backward, for xbar = dL/dx: lambda = M^{-1} xbar by a second
BRAS-PCG solve (M is symmetric), so bbar = lambda, and zbar_K = rho_K rhobar_K =
-rho_K lambda_K^T M_K^1 x_K from the library's fused element kernel.  All numerical work runs
in libbras; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import bras as B


class BrasMassSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, b, solver: "WeightedMassSolver"):
        x = solver._solve(z.detach(), b.detach())
        ctx.solver = solver
        ctx.save_for_backward(z.detach(), x)
        return x

    @staticmethod
    def backward(ctx, xbar):
        z, x = ctx.saved_tensors
        solver = ctx.solver
        lam = solver._solve(z, xbar.contiguous().to(torch.float64))
        return solver.context.grad_log_rho(x, lam), lam, None


class WeightedMassSolver:
    """Holds one H1 context; ``__call__(z, b)`` is differentiable in z and b."""

    def __init__(self, coords, cells, order, n_dof, l2g, rtol=1e-12, mode=B.SOLVE_FP64, maxit=5000, space="h1"):
        self.context = B.Context(coords, cells, space, order, n_dof, l2g)
        self.rtol, self.mode, self.maxit = rtol, mode, maxit
        self.last = None

    def _solve(self, z, b):
        self.context.update_log_rho(z.to(torch.float64))
        x, its, rel, st = self.context.pcg_solve(b.contiguous(), pc=B.PC_BRAS, mode=self.mode, rtol=self.rtol,
                                                 maxit=self.maxit)
        if st != B.OK:
            raise B.BrasError(st if st < 0 else -8, "weighted mass solve did not converge")
        self.last = (int(its[0]), float(rel[0]))
        return x

    def __call__(self, z, b):
        return BrasMassSolve.apply(z, b, self)
