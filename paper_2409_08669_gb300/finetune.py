"""Load-balancing fine-tune (Sec. 4.4, the total loss): optimise the Gaussians
of a scene against target images under

    L = lambda_L1 * L1 + lambda_ssim * (1 - SSIM) + lambda_load * L_load,

lambda_L1 + lambda_ssim + lambda_load = 1, with lambda_load = 0.45 and the
remaining 0.55 split 4:1 between L1 and SSIM (the 0.8 / 0.2 weighting of the
3DGS objective the paper starts from).  L_load (Eq. 13) is the standard
deviation over the pixels of the per-pixel load l_i (Eq. 12).  The paper gives
no derivative of the integer count l_i; the settings pick the reading: the
straight-through one (d l_i / d alpha_k = 1 for every Gaussian blended into the
pixel) or the termination one (for a pixel that stopped early,
d l_i / d alpha_k = -l_i / (-ln T_final) / (1 - alpha_k): a more opaque Gaussian
brings the stop forward and shortens l_i).

Every loss term and every gradient of the rasterizer runs in libadr.so
(adr_render / adr_render_backward, adr_image_loss, adr_load_loss); PyTorch
holds the raw parameters, applies the activations (exp of the log-scales,
sigmoid of the opacity logits) and runs Adam.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from .autograd import l1_ssim_loss, load_balance_loss, rasterize
from .raster import Rasterizer, image_loss, upload


@dataclasses.dataclass
class FinetuneConfig:
    steps: int = 300
    lambda_l1: float = 0.44
    lambda_ssim: float = 0.11
    lambda_load: float = 0.45
    # Adam step sizes per parameter group: a fifth of the 3DGS defaults
    # (positions in world units for a scene of extent ~10), for a short
    # fine-tune of an already fitted scene
    lr_means: float = 3.2e-6
    lr_log_scales: float = 1e-3
    lr_rots: float = 2e-4
    lr_opacity_logits: float = 5e-3
    lr_sh: float = 5e-4


class Finetuner:
    """Holds the raw parameters of a scene and steps the total loss over a
    cycle of (camera, target image) pairs."""

    def __init__(self, scene, cameras, targets, rast: Rasterizer, settings, cfg: FinetuneConfig):
        means, scales, rots, opac, sh = upload(scene, f"cuda:{rast.device}")
        self.raw = [means.clone().requires_grad_(True),
                    torch.log(scales).requires_grad_(True),
                    rots.clone().requires_grad_(True),
                    torch.logit(opac.clamp(1e-4, 1 - 1e-4)).requires_grad_(True),
                    sh.clone().requires_grad_(True)]
        lrs = (cfg.lr_means, cfg.lr_log_scales, cfg.lr_rots, cfg.lr_opacity_logits, cfg.lr_sh)
        self.opt = torch.optim.Adam([{"params": [p], "lr": lr} for p, lr in zip(self.raw, lrs)],
                                    eps=1e-15)
        self.cameras, self.targets = cameras, targets
        self.rast, self.settings, self.cfg = rast, settings, cfg
        self.k = 0

    def params(self):
        """Activated parameters (means, scales, rots, opacity, sh)."""
        r = self.raw
        return (r[0], torch.exp(r[1]), r[2], torch.sigmoid(r[3]), r[4])

    def step(self):
        """One iteration; returns the loss tensor (device, not synchronised)."""
        cfg = self.cfg
        i = self.k % len(self.cameras)
        self.k += 1
        self.opt.zero_grad(set_to_none=True)
        img, load_f, _ = rasterize(self.params(), self.rast, self.cameras[i], self.settings)
        loss = l1_ssim_loss(img, self.targets[i], cfg.lambda_l1, cfg.lambda_ssim)
        if cfg.lambda_load > 0.0:
            loss = loss + cfg.lambda_load * load_balance_loss(load_f, self.rast)
        loss.backward()
        self.opt.step()
        return loss.detach()

    def activated_copy(self):
        with torch.no_grad():
            return tuple(t.detach().contiguous().clone() for t in self.params())


def render_targets(rast: Rasterizer, params, cameras, settings):
    out = []
    for cam in cameras:
        img, _, _ = rast.forward(params, cam, settings, want_aux=False)
        out.append(img.clone())
    torch.cuda.synchronize(rast.device)
    return out


def evaluate(rast: Rasterizer, params, cameras, targets, settings, repeats=5):
    """Frames/s of the whole frame (preprocess + sort + render, CUDA events over
    `repeats` passes of the cameras, without depth slices so that the frame's
    work does not depend on the context's slicing history), mean and std of
    the per-pixel load l_i, and PSNR / SSIM against the targets, averaged over
    the cameras."""
    rast.set_depth_slices(Rasterizer.SLICES_NEVER)
    stds, means, psnr, ssim = [], [], [], []
    for cam, tgt in zip(cameras, targets):
        img, _, load = rast.forward(params, cam, settings)
        stats, _ = rast.load_loss(load, want_grad=False)
        st, _ = image_loss(img, tgt, want_grad=False)
        mse = float(((img - tgt) ** 2).mean())
        stats, st = stats.cpu(), st.cpu()
        means.append(float(stats[0]))
        stds.append(float(stats[1]))
        ssim.append(float(st[1]))
        psnr.append(10.0 * math.log10(1.0 / max(mse, 1e-20)))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for cam in cameras:                      # warm-up
        rast.forward(params, cam, settings, want_aux=False)
    torch.cuda.synchronize(rast.device)
    ev0.record()
    for _ in range(repeats):
        for cam in cameras:
            rast.forward(params, cam, settings, want_aux=False)
    ev1.record()
    torch.cuda.synchronize(rast.device)
    rast.set_depth_slices(Rasterizer.SLICES_ADAPTIVE)
    frames = repeats * len(cameras)
    k = len(cameras)
    return {"fps": frames * 1e3 / ev0.elapsed_time(ev1), "load_mean": sum(means) / k,
            "load_std": sum(stds) / k, "psnr_db": sum(psnr) / k, "ssim": sum(ssim) / k}
