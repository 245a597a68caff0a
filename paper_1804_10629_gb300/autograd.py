"""Differentiable enlarged solve: torch.autograd Functions around the C-ABI library.

Forward: x = A^{-1} b by the s-step enlarged CG.  Backward: A is SPD, so the adjoint system
A lambda = dL/dx is a second enlarged solve on the same context; then dL/db = lambda and
dL/dA_ij = -lambda_i x_j on the sparsity pattern, chained to the coefficient field of the
2D diffusion model by a library kernel.  Only x (and the inputs) are kept for the backward
pass, not the Krylov basis.  Every vector operation runs in libekcg's kernels; torch holds
the device memory.
"""
from __future__ import annotations

import torch

from . import ekcg


def _solve(solver, rhs, s, tol, maxit):
    x, it, hist, st = solver.solve(rhs.contiguous(), s=s, tol=tol, maxit=maxit)
    if st not in (ekcg.EKCG_OK,):
        raise ekcg.EkcgError(st, "enlarged solve in autograd")
    return x


class EnlargedSolve(torch.autograd.Function):
    """x = A(val)^{-1} b, differentiable in b and in the CSR values `val` of A."""

    @staticmethod
    def forward(ctx, b, val, solver, s, tol, maxit):
        ekcg.ekcg_update_values(solver.ctx, val.contiguous())
        x = _solve(solver, b, s, tol, maxit)
        ctx.solver, ctx.s, ctx.tol, ctx.maxit = solver, s, tol, maxit
        ctx.save_for_backward(x, val)
        return x

    @staticmethod
    def backward(ctx, gx):
        x, val = ctx.saved_tensors
        solver = ctx.solver
        ekcg.ekcg_update_values(solver.ctx, val.contiguous())
        lam = _solve(solver, gx, ctx.s, ctx.tol, ctx.maxit)
        dval = None
        if ctx.needs_input_grad[1]:
            dval = torch.empty_like(val)
            ekcg.ekcg_grad_A(solver.ctx, lam, x, dval)
        return lam, dval, None, None, None, None


class Diffusion2DSolve(torch.autograd.Function):
    """x = A(kappa)^{-1} b for the 2D edge-form diffusion model, kappa = exp(log_kappa);
    differentiable in log_kappa and b."""

    @staticmethod
    def forward(ctx, log_kappa, b, solver, nx, ny, ax, ay, s, tol, maxit):
        lk = log_kappa.contiguous()
        val = torch.empty(solver.nnz, dtype=torch.float64, device=b.device)
        ekcg.ekcg_diffusion2d_values(solver.ctx, nx, ny, ax, ay, lk, val)
        ekcg.ekcg_update_values(solver.ctx, val)
        x = _solve(solver, b, s, tol, maxit)
        ctx.solver = solver
        ctx.args = (nx, ny, ax, ay, s, tol, maxit)
        ctx.save_for_backward(lk, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        lk, x = ctx.saved_tensors
        nx, ny, ax, ay, s, tol, maxit = ctx.args
        solver = ctx.solver
        val = torch.empty(solver.nnz, dtype=torch.float64, device=x.device)
        ekcg.ekcg_diffusion2d_values(solver.ctx, nx, ny, ax, ay, lk, val)
        ekcg.ekcg_update_values(solver.ctx, val)
        lam = _solve(solver, gx, s, tol, maxit)
        glk = torch.empty_like(lk)
        ekcg.ekcg_diffusion2d_grad_logkappa(solver.ctx, nx, ny, ax, ay, lk, lam, x, glk)
        return glk, lam, None, None, None, None, None, None, None, None


def enlarged_solve(b, val, solver, s=2, tol=1e-10, maxit=10000):
    return EnlargedSolve.apply(b, val, solver, s, tol, maxit)


def diffusion2d_solve(log_kappa, b, solver, nx, ny, ax=1.0, ay=1.0, s=3, tol=1e-10,
                      maxit=10000):
    return Diffusion2DSolve.apply(log_kappa, b, solver, nx, ny, ax, ay, s, tol, maxit)
