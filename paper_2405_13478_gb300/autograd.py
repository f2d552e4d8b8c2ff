"""torch.autograd wrappers of the imaging path and its adjoint.

``dirty_images(vis, plan)`` images complex64 visibilities with the plan's
kernels; its backward runs the library's adjoint kernels (forward FFT of the
image gradient + degridding, ``blink_plan_degrid``), recomputing from the
plan instead of storing grids.  ``image_sqnorm(vis, plan, ...)`` returns
each layer's sum of squares of the (residual) image, formed by the fused
epilogue as the image is stored, and keeps the adjoint's column transforms
of the stored image (``blink_epilogue.d_adjoint``); its backward finishes the
adjoint from those with a per-layer factor (``blink_plan_degrid_adjoint``),
so no image-sized gradient is formed and the images are not read again.  ``apply_gains(gains, model, ...)`` forms
V_ij = g_i conj(g_j) M_ij with ``blink_apply_gains``; its backward is
``blink_gain_grad``.  Gradients follow torch's complex convention
dL/dRe + i dL/dIm.  No image-sized computation happens in torch: it
allocates the tensors, carries the graph and forms per-layer factors.
"""
from __future__ import annotations

import torch

from . import binding


class _DirtyImages(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis, plan, n_out, flags, ref):
        if vis.dtype != torch.complex64 or not vis.is_cuda:
            raise ValueError("vis must be a complex64 CUDA tensor")
        vis = vis.contiguous()
        out = torch.empty(n_out, dtype=torch.float32, device=vis.device)
        if ref is None:
            plan.image(vis, out, None, flags)
        else:  # the fused epilogue subtracts the constant reference at the store
            plan.image(vis, out, None, flags, ref=ref.detach().contiguous())
        ctx.plan = plan
        ctx.flags = flags
        ctx.vis_shape = vis.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        grad_out = grad_out.contiguous()
        dvis = torch.zeros(ctx.vis_shape, dtype=torch.complex64, device=grad_out.device)
        ctx.plan.degrid(grad_out, dvis, ctx.flags)
        return dvis, None, None, None, None


def dirty_images(vis: torch.Tensor, plan: "binding.Plan", n_out: int, flags: int = 0,
                 ref: torch.Tensor | None = None):
    """Float32 images (packed at the plan's out_offsets, ``n_out`` floats).
    With ``ref`` (float32, laid out like the images, no gradient) the result
    is image - ref, subtracted by the fused epilogue as the images are
    stored; the gradient with respect to the visibilities is the same."""
    return _DirtyImages.apply(vis, plan, n_out, flags, ref)


class _ImageSqNorm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis, plan, n_out, flags, ref):
        if vis.dtype != torch.complex64 or not vis.is_cuda:
            raise ValueError("vis must be a complex64 CUDA tensor")
        vis = vis.contiguous()
        sq = torch.empty(plan.n_layers, dtype=torch.float64, device=vis.device)
        adj = torch.empty(plan.adjoint_bytes() // 4, dtype=torch.float32, device=vis.device)
        # no image array: the residual is summed and column-transformed as it
        # is formed, never stored
        plan.image(vis, None, None, flags, ref=None if ref is None else ref.detach().contiguous(), sqnorm=sq,
                   adjoint=adj)
        ctx.plan, ctx.flags, ctx.vis_shape = plan, flags, vis.shape
        # the residual's column transforms: dL/dI_l = 2 dL/ds_l * resid_l
        ctx.adj = adj
        return sq

    @staticmethod
    def backward(ctx, grad_sq):
        scale = (2.0 * grad_sq).to(torch.float32).contiguous()
        dvis = torch.zeros(ctx.vis_shape, dtype=torch.complex64, device=grad_sq.device)
        ctx.plan.degrid_adjoint(ctx.adj, dvis, ctx.flags, layer_scale=scale)
        return dvis, None, None, None, None


def image_sqnorm(vis: torch.Tensor, plan: "binding.Plan", n_out: int, flags: int = 0,
                 ref: torch.Tensor | None = None):
    """Float64 [layers]: layer l's sum over its pixels of (image - ref)^2
    (of the image alone without ``ref``), summed by the fused epilogue as the
    image is formed (no image is stored: the backward starts from the
    adjoint's column transforms of the residual, r_alloc x N complex values
    per layer; ``n_out`` is accepted for symmetry with dirty_images).  A least-squares image loss is ``image_sqnorm(...).sum()``."""
    return _ImageSqNorm.apply(vis, plan, n_out, flags, ref)


class _ApplyGains(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, model, lib_ctx, n_ant, layers):
        if gains.dtype != torch.complex64 or model.dtype != torch.complex64:
            raise ValueError("gains and model must be complex64")
        gains = gains.contiguous()
        model = model.contiguous()
        vis = torch.empty_like(model)
        lib_ctx.apply_gains(n_ant, layers, model, gains, vis)
        ctx.save_for_backward(gains, model)
        ctx.lib_ctx, ctx.n_ant, ctx.layers = lib_ctx, n_ant, layers
        return vis

    @staticmethod
    def backward(ctx, grad_vis):
        gains, model = ctx.saved_tensors
        dg = torch.empty_like(gains)
        ctx.lib_ctx.gain_grad(ctx.n_ant, ctx.layers, grad_vis.contiguous(), model, gains, dg)
        return dg, None, None, None, None


def apply_gains(gains: torch.Tensor, model: torch.Tensor, lib_ctx: "binding.Context", n_ant: int,
                layers):
    """V_ij = g_i conj(g_j) M_ij for every layer (vis_offset addressing)."""
    return _ApplyGains.apply(gains, model, lib_ctx, n_ant, layers)
