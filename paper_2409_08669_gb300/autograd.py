"""torch.autograd glue over the C ABI (argument marshalling only).

AdrRasterize: forward = adr_preprocess + adr_sort + adr_render, backward =
adr_render_backward.  Outputs the image and the per-pixel load l_i (Eq. 12)
as a float tensor; a gradient reaching the load flows back through the
reading settings.load_grad selects (straight-through d l_i / d alpha = 1, or
the early-stop reading for pixels that terminated; Sec. 4.4).
LoadBalanceLoss: L_load = std of l_i over the pixels (Eq. 13), computed and
differentiated by adr_load_loss.
ImageLoss: w_l1 * L1 + w_ssim * (1 - SSIM) against a target image, computed and
differentiated by adr_image_loss (the L1 and SSIM terms of the total loss).
"""
from __future__ import annotations

import torch

from .raster import Rasterizer, image_loss


class AdrRasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, rots, opac, sh, rast: Rasterizer, camera, settings):
        params = tuple(t.contiguous() for t in (means, scales, rots, opac, sh))
        img, t_final, load = rast.forward(params, camera, settings)
        ctx.rast = rast
        ctx.frame = rast.frame
        ctx.save_for_backward(*params)
        ctx.load_int = load
        ctx.mark_non_differentiable(t_final)
        return img, load.to(torch.float32), t_final

    @staticmethod
    def backward(ctx, g_img, g_load, g_t):
        params = ctx.saved_tensors
        if ctx.rast.frame != ctx.frame:
            raise RuntimeError("the Rasterizer rendered another frame before this backward; "
                               "use one Rasterizer per frame in flight")
        if g_img is None:
            g_img = torch.zeros((3,) + ctx.load_int.shape, device=params[0].device)
        grads = ctx.rast.backward(params, g_img, g_load)
        return (*grads, None, None, None)


class LoadBalanceLoss(torch.autograd.Function):
    """std over pixels of the load; input is the float load from AdrRasterize."""

    @staticmethod
    def forward(ctx, load_f, rast: Rasterizer):
        load_i = load_f.detach().round().to(torch.int32)
        stats, grad = rast.load_loss(load_i, 1.0, want_grad=True)
        ctx.save_for_backward(grad)
        return stats[1].to(torch.float32)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


class ImageLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, ref, w_l1, w_ssim):
        stats, grad = image_loss(img.detach(), ref.detach(), w_l1, w_ssim, want_grad=True)
        ctx.save_for_backward(grad)
        ctx.stats = stats
        return (w_l1 * stats[0] + w_ssim * (1.0 - stats[1])).to(torch.float32)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None, None


def rasterize(params, rast: Rasterizer, camera, settings):
    """(img [3,H,W], load [H,W] float, t_final [H,W]) differentiable w.r.t. params."""
    return AdrRasterize.apply(*params, rast, camera, settings)


def load_balance_loss(load_f, rast: Rasterizer):
    return LoadBalanceLoss.apply(load_f, rast)


def l1_ssim_loss(img, ref, w_l1=0.8, w_ssim=0.2):
    """w_l1 * mean|img - ref| + w_ssim * (1 - SSIM(img, ref)), differentiable in img."""
    return ImageLoss.apply(img, ref, float(w_l1), float(w_ssim))
