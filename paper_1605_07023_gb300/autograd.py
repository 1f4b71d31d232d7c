"""torch.autograd wrappers: grid() with degridding as its hand-written backward.

Gridding is linear in the visibilities: grid = A diag(w) v, where A holds the
real separable taps (Sec. 2.2, Sec. 4). For a real loss, PyTorch passes
dL/d(out)* to backward, and the gradient of a linear map is its Hermitian
adjoint applied to that. So:
  - d/dv of grid():   grad_v = diag(w) A^T grad_grid = degrid_weighted(grad_grid, w)
  - d/dg of degrid(): grad_g = A grad_v                = grid(grad_v, unit weights)
Both run in the library's CUDA kernels. The forward map and its backward are
the exact adjoint pair that the oracle's adjoint test pins.
"""
from __future__ import annotations

import torch

from . import Plan, degrid, degrid_weighted, grid


class GridFn(torch.autograd.Function):
    """vis [n, P] complex64 -> grid [P, G, G] complex64 (fresh, zero-initialised)."""

    @staticmethod
    def forward(ctx, vis, uv, weights, table, plan: Plan):
        if plan.precision != "f32":
            raise ValueError("autograd needs an FP32 plan")
        g = torch.zeros((plan.npol, plan.G, plan.G), dtype=torch.complex64, device=vis.device)
        grid(plan, uv, vis.contiguous(), weights, table, g)
        ctx.plan = plan
        ctx.save_for_backward(uv, weights, table)
        return g

    @staticmethod
    def backward(ctx, grad_grid):
        uv, weights, table = ctx.saved_tensors
        gv = None
        if ctx.needs_input_grad[0]:
            gv = degrid_weighted(ctx.plan, uv, grad_grid.contiguous(), table, weights)
        return gv, None, None, None, None


class DegridFn(torch.autograd.Function):
    """grid [P, G, G] complex64 -> vis [n, P] complex64."""

    @staticmethod
    def forward(ctx, g, uv, table, plan: Plan):
        v = degrid(plan, uv, g.contiguous(), table)
        ctx.plan = plan
        ctx.save_for_backward(uv, table)
        return v

    @staticmethod
    def backward(ctx, grad_vis):
        uv, table = ctx.saved_tensors
        gg = None
        if ctx.needs_input_grad[0]:
            gg = torch.zeros((ctx.plan.npol, ctx.plan.G, ctx.plan.G), dtype=torch.complex64, device=grad_vis.device)
            grid(ctx.plan, uv, grad_vis.contiguous(), None, table, gg)
        return gg, None, None, None


def grid_op(plan: Plan, uv, vis, weights, table):
    """Differentiable grid(): returns a fresh [P, G, G] grid; the gradient flows to vis."""
    return GridFn.apply(vis, uv, weights, table, plan)


def degrid_op(plan: Plan, uv, g, table):
    """Differentiable degrid(): returns [n, P] visibilities; the gradient flows to the grid."""
    return DegridFn.apply(g, uv, table, plan)
