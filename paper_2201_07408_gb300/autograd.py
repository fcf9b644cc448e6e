"""torch.autograd Functions over the C-ABI.

ProjectA:      y = A x; backward dL/dx = A^T dL/dy with the exact-transpose
               kernel (Sec. I, Eq. 3 uses A^T).
BAGMRESSolve:  x = (BA)^{-1} B b, the converged BA-GMRES solution (Sec. II,
               Eq. 5); backward dL/db = B^T (A^T B^T)^{-1} dL/dx by GMRES on
               A^T B^T (ct_bagmres_vjp).  The derivative is that of the
               converged solution (the implicit-function derivative), so the
               forward solve should be run to a small tolerance.  The forward
               Krylov basis is not kept: the backward builds its own.
"""
from __future__ import annotations

import torch

from . import ct


class ProjectA(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, geom):
        ctx.geom = geom
        return ct.project_A(geom, x.detach().contiguous())

    @staticmethod
    def backward(ctx, gy):
        return ct.adjoint_At(ctx.geom, gy.contiguous()), None


class BAGMRESSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, geom, k, b_kind, tol, k_adjoint, tol_adjoint):
        x, res = ct.bagmres(geom, b.detach().contiguous(), k, b_kind=b_kind, tol=tol)
        ctx.geom, ctx.b_kind = geom, b_kind
        ctx.k_adjoint, ctx.tol_adjoint = k_adjoint, tol_adjoint
        ctx.forward_result = res
        return x

    @staticmethod
    def backward(ctx, gx):
        geom = ctx.geom
        gb = torch.empty(geom.sino_shape, dtype=torch.float32, device=geom.device)
        res = ct.ct_bagmres_vjp(geom, gx.contiguous(), ctx.k_adjoint, gb,
                                ct.make_opts(b_kind=ctx.b_kind, tol=ctx.tol_adjoint))
        ctx.adjoint_result = res
        return gb, None, None, None, None, None, None


def project_A(geom, x):
    """Differentiable y = A x."""
    return ProjectA.apply(x, geom)


def bagmres_solve(geom, b, k=200, b_kind="un", tol=1e-6, k_adjoint=None, tol_adjoint=None):
    """Differentiable converged BA-GMRES solve x = (BA)^{-1} B b."""
    return BAGMRESSolve.apply(b, geom, k, b_kind, tol, k if k_adjoint is None else k_adjoint,
                              tol if tol_adjoint is None else tol_adjoint)
