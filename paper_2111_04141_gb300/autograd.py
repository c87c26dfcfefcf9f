"""Differentiable gridding and degridding (torch.autograd.Function).

Gridding G (visibilities -> grid) and degridding G^H (grid -> visibilities)
are linear maps that are each other's adjoint, so each is the hand-written
backward of the other: for y = G v the vector-Jacobian product is
grad_v = G^H grad_y (a degridding call), and for v = G^H g it is
grad_g = G grad_v (a gridding call).  The correction and the origin shift
are real diagonal operators, their own adjoints.  Every forward and
backward step runs in libgw's CUDA kernels; the FFTs between grid and
image are cuFFT calls through torch.fft.

Imaging operators (the thesis' imaging chain, Section 2.3, and its adjoint):

  dirty(v)   = correct(+1)( IFFT( shift( G v ) ) )    visibilities -> image
  predict(x) = G^H( shift( FFT( correct(-1)(x) ) ) )  image -> visibilities

with unnormalised transforms, so that predict is exactly the adjoint of
dirty.  Plans must use complex64 storage (c64 tables and visibilities).
"""
from __future__ import annotations

import torch


def _check(plan):
    if plan.vis_dtype != "c64":
        raise ValueError("autograd needs a plan with complex64 visibilities (vis_dtype='c64')")


class GridFn(torch.autograd.Function):
    """grid = G vis; backward: grad_vis = G^H grad_grid (degridding)."""

    @staticmethod
    def forward(ctx, vis, plan, uvw, freq):
        _check(plan)
        ctx.plan, ctx.uvw, ctx.freq = plan, uvw, freq
        return plan.grid(uvw, freq, vis.contiguous())

    @staticmethod
    def backward(ctx, grad_grid):
        g = None
        if ctx.needs_input_grad[0]:
            g = ctx.plan.degrid(ctx.uvw, ctx.freq, grad_grid.contiguous())
        return g, None, None, None


class DegridFn(torch.autograd.Function):
    """vis = G^H grid; backward: grad_grid = G grad_vis (gridding)."""

    @staticmethod
    def forward(ctx, grid, plan, uvw, freq):
        _check(plan)
        ctx.plan, ctx.uvw, ctx.freq = plan, uvw, freq
        return plan.degrid(uvw, freq, grid.contiguous())

    @staticmethod
    def backward(ctx, grad_vis):
        g = None
        if ctx.needs_input_grad[0]:
            g = ctx.plan.grid(ctx.uvw, ctx.freq, grad_vis.contiguous())
        return g, None, None, None


class CorrectFn(torch.autograd.Function):
    """Grid correction (real diagonal, self-adjoint) with the given direction."""

    @staticmethod
    def forward(ctx, image, plan, direction):
        ctx.plan, ctx.direction = plan, direction
        return plan.correct(image.contiguous().clone(), direction=direction)

    @staticmethod
    def backward(ctx, grad):
        g = None
        if ctx.needs_input_grad[0]:
            g = ctx.plan.correct(grad.contiguous().clone(), direction=ctx.direction)
        return g, None, None


class ShiftFn(torch.autograd.Function):
    """Origin shift (-1)^(kv + ku) (real diagonal, self-adjoint)."""

    @staticmethod
    def forward(ctx, grid, plan):
        ctx.plan = plan
        return plan.shift(grid.contiguous().clone())

    @staticmethod
    def backward(ctx, grad):
        g = None
        if ctx.needs_input_grad[0]:
            g = ctx.plan.shift(grad.contiguous().clone())
        return g, None


def grid(plan, uvw, freq, vis):
    return GridFn.apply(vis, plan, uvw, freq)


def degrid(plan, uvw, freq, grid_):
    return DegridFn.apply(grid_, plan, uvw, freq)


def dirty(plan, uvw, freq, vis):
    """[npol, N, N] dirty image of visibilities [nrow, nchan, npol]."""
    g = ShiftFn.apply(GridFn.apply(vis, plan, uvw, freq), plan)
    img = torch.fft.ifft2(g, norm="forward")          # unnormalised inverse transform
    return CorrectFn.apply(img, plan, +1)


def predict(plan, uvw, freq, image):
    """Model visibilities [nrow, nchan, npol] of a [npol, N, N] image (real or
    complex); the adjoint of ``dirty``."""
    if not image.is_complex():
        image = torch.complex(image, torch.zeros_like(image))
    x = CorrectFn.apply(image.to(torch.complex64), plan, -1)
    g = ShiftFn.apply(torch.fft.fft2(x, norm="backward"), plan)   # unnormalised forward
    return DegridFn.apply(g, plan, uvw, freq)


def chisq(plan, uvw, freq, sky, data, sigma):
    """sum |predict(sky) - data|^2 / sigma^2, summed in float64."""
    r = predict(plan, uvw, freq, sky) - data
    return (torch.view_as_real(r).double() ** 2).sum() / (sigma * sigma)
