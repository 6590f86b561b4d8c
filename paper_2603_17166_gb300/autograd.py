"""torch.autograd wrappers of a plan's synthesis and adjoint.

Synthesis general is real-linear in (g, c), so its backward pass is the adjoint and the adjoint's
backward pass is the synthesis.  torch's gradient of a real loss with respect to a complex tensor
is dL/dRe + i dL/dIm over the stored entries; the packed a_lm arrays store m >= 0 only, each
m > 0 entry standing for the pair (m, -m) tied by the reality condition of eq. syn.  The library's
packed-gradient entry points (psht_plan_adjoint_packed, psht_plan_synthesis_packed) apply that
factor of two inside the recursion kernels, so both passes are one library call each.
"""
from __future__ import annotations

import torch

from .psht import Plan, nalm


class _Synthesis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, c, plan):
        ctx.plan = plan
        ctx.g_dtype = g.dtype
        ctx.c_dtype = None if c is None else c.dtype
        return plan.synthesis(g, c)

    @staticmethod
    def backward(ctx, grad_f):
        want_c = ctx.c_dtype is not None and ctx.needs_input_grad[1]
        gg, gc = ctx.plan.adjoint(grad_f.contiguous(), want_c=want_c, packed_grad=True)
        gg = gg.to(ctx.g_dtype) if ctx.needs_input_grad[0] else None
        gc = gc.to(ctx.c_dtype) if want_c else None
        return gg, gc, None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan, want_c):
        ctx.plan = plan
        ctx.f_dtype = f.dtype
        g, c = plan.adjoint(f, want_c=want_c)
        return (g, c) if want_c else (g,)

    @staticmethod
    def backward(ctx, grad_g, *rest):
        grad_c = rest[0] if rest else None
        plan = ctx.plan
        if grad_g is None:
            grad_g = torch.zeros(nalm(plan.lmax), dtype=plan.cdtype, device="cuda")
        gf = plan.synthesis(grad_g.contiguous(), None if grad_c is None else grad_c.contiguous(), packed_grad=True)
        return gf.to(ctx.f_dtype), None, None


def synthesis(plan: Plan, g: torch.Tensor, c: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable f = synthesis(g, c) at the plan's points."""
    return _Synthesis.apply(g, c, plan)


def adjoint(plan: Plan, f: torch.Tensor, want_c: bool = True):
    """Differentiable (g~, c~) = adjoint(f) at the plan's points; (g~,) when want_c is False."""
    out = _Adjoint.apply(f, plan, want_c)
    return out if want_c else out[0]
