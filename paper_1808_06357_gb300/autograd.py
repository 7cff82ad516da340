"""torch.autograd.Function around the Strang evolution and its adjoint.

`strang_evolve(plan, v, u0, dt, nsteps)` returns u_N = S(dt)^nsteps u0 computed
by the library's kernels; its backward pass calls lsp_adjoint (the
conjugate-transposed step run backward, with checkpoints) for the gradients
with respect to the potential samples v and the initial state u0.  Complex
gradients follow PyTorch's convention for a real loss: dL/dRe + i dL/dIm.
"""

from __future__ import annotations

import torch

from ._binding import Plan, adjoint


class StrangEvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, u0, plan: Plan, dt: float, nsteps: int, ckpt_stride: int = 0):
        plan.set_potential(v.contiguous())
        plan.set_state(u0.contiguous())
        plan.strang_steps(dt, nsteps)
        out = plan.get_state(prec="c64" if u0.dtype == torch.complex64 else "c128")
        ctx.save_for_backward(v, u0)
        ctx.plan, ctx.dt, ctx.nsteps, ctx.ckpt = plan, dt, nsteps, ckpt_stride
        return out

    @staticmethod
    def backward(ctx, g_out):
        v, u0 = ctx.saved_tensors
        plan = ctx.plan
        plan_dtype = torch.complex64 if plan.prec == 1 else torch.complex128
        lam = g_out.resolve_conj().resolve_neg().to(plan_dtype).contiguous()
        grad_v = torch.empty_like(v, dtype=torch.float64)
        grad_u0 = torch.empty(u0.numel(), dtype=plan_dtype, device=u0.device)
        plan.set_potential(v.contiguous())
        plan.set_state(u0.contiguous())
        adjoint(plan, ctx.dt, ctx.nsteps, lam, grad_v, grad_u0, ctx.ckpt)
        return grad_v.to(v.dtype), grad_u0.to(u0.dtype), None, None, None, None


def strang_evolve(plan: Plan, v, u0, dt: float, nsteps: int, ckpt_stride: int = 0):
    """u_N = S(dt)^nsteps u0 on `plan`, differentiable in v (float64) and u0 (complex)."""
    return StrangEvolve.apply(v, u0, plan, dt, nsteps, ckpt_stride)
