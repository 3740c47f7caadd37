"""torch.autograd.Function over the C ABI: the NeuRLP-PDE layer.

Forward (Eqs. 9-10): z* = argmin ||A z - d|| for the PDE data (coefficient
fields and per-instance scalars, right-hand side b, Dirichlet values omega).
Backward (Eq. 11 and the gradients after it): one adjoint solve with the same
operator gives dl/dfields, dl/dscalars, dl/db and dl/domega.  With
``recompute=True`` the forward solution is not kept for the backward pass;
the adjoint call recomputes it (less memory, one more solve).  Without it,
the backward pass reuses the problem's kept forward state only if no other
forward ran on the same solver in between (its generation counter is
unchanged); otherwise it recomputes, so interleaved solves never mix states.
"""
from __future__ import annotations

import torch

from .binding import Solver


class NeuRLPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fields, scalars, rhs, omega, solver: Solver, recompute: bool = False):
        fields_c = fields.contiguous()
        scalars_c = scalars.contiguous()
        rhs_c = rhs.contiguous()
        omega_c = omega.contiguous()
        z = solver.forward(fields_c, scalars_c, rhs_c, omega_c)
        ctx.solver = solver
        ctx.recompute = recompute
        ctx.gen = solver.generation()
        if recompute:
            ctx.save_for_backward(fields_c, scalars_c, rhs_c, omega_c)
        else:
            ctx.save_for_backward(fields_c, scalars_c, rhs_c, omega_c, z)
        return z

    @staticmethod
    def backward(ctx, g_z):
        saved = ctx.saved_tensors
        fields, scalars, rhs, omega = saved[:4]
        z = None if ctx.recompute else saved[4]
        reuse = not ctx.recompute and ctx.solver.generation() == ctx.gen
        dfields, dscal, drhs, dom = ctx.solver.adjoint(fields, scalars, rhs, omega, z, g_z.contiguous(),
                                                       reuse_setup=reuse)
        return dfields, dscal, drhs, dom, None, None


def solve(fields, scalars, rhs, omega, solver: Solver, recompute: bool = False):
    """Differentiable batched solve: returns z [B][V][N]."""
    return NeuRLPSolve.apply(fields, scalars, rhs, omega, solver, recompute)
