"""Rasterizer: device-tensor wrapper over the C ABI (marshalling only).

PyTorch provides device memory and streams; every stage runs in libadr.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .scenes import Scene

TILE = _lib.ADR_TILE


def upload(scene: Scene, device="cuda") -> tuple:
    """Copy a scene's arrays to device float32 tensors (means, scales, rots, opac, sh)."""
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in scene.arrays())


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# values per Gaussian of (means, scales, rots, opacity, SH) in the C ABI's layout
PARAM_NAMES = ("means", "scales", "rots", "opac", "sh")
PARAM_WIDTHS = (3, 3, 4, 1, 48)


def check_tensor(name, t, numel, dtype=torch.float32, device=None):
    """Raise unless `t` is a contiguous `dtype` tensor of `numel` values (on
    cuda:`device` when given): the kernels read and write exactly that many
    values behind the pointer, so a mismatch must not reach them."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} holds {t.numel()} values, expected {numel}")
    if device is not None and (not t.is_cuda or t.device.index != device):
        raise ValueError(f"{name} must be on cuda:{device}, got {t.device}")


def check_params(params, device=None):
    """Validates (means [n,3], scales [n,3], rots [n,4], opac [n], sh [n,16,3]),
    float32 and contiguous (on cuda:`device` when given); returns n."""
    if len(params) != 5:
        raise ValueError(f"expected 5 parameter tensors, got {len(params)}")
    means = params[0]
    if not isinstance(means, torch.Tensor) or means.dim() != 2 or means.shape[1] != 3:
        raise ValueError("means must be an [n, 3] tensor")
    n = int(means.shape[0])
    for name, t, width in zip(PARAM_NAMES, params, PARAM_WIDTHS):
        check_tensor(name, t, width * n, device=device)
    return n


def image_loss(img, ref, w_l1=1.0, w_ssim=0.0, want_grad=True, stream=None, scratch=None):
    """(stats, grad): stats = device float64 [mean |img - ref|, mean SSIM] and
    grad = d(w_l1 * L1 + w_ssim * (1 - SSIM)) / d img (None unless want_grad),
    computed by adr_image_loss.  img, ref: [C, H, W] float32 on one device."""
    img, ref = img.contiguous(), ref.contiguous()
    if img.dim() != 3:
        raise ValueError(f"img must be [C, H, W], got shape {tuple(img.shape)}")
    if ref.shape != img.shape:
        raise ValueError(f"ref shape {tuple(ref.shape)} differs from img {tuple(img.shape)}")
    if not img.is_cuda:
        raise ValueError(f"img must be a CUDA tensor, got {img.device}")
    check_tensor("img", img, img.numel(), device=img.device.index)
    check_tensor("ref", ref, img.numel(), device=img.device.index)
    c, h, w = img.shape
    stats = torch.empty(2, dtype=torch.float64, device=img.device)
    grad = None
    if want_grad:
        grad = torch.empty_like(img)
        if scratch is None or scratch.numel() < 3 * img.numel():
            scratch = torch.empty(3 * img.numel(), dtype=torch.float32, device=img.device)
    with torch.cuda.device(img.device):
        _lib.adr_image_loss(_ptr(img), _ptr(ref), c, h, w, float(w_l1), float(w_ssim), _ptr(stats),
                            _ptr(grad), _ptr(scratch) if want_grad else 0, _stream(stream))
    return stats, grad


class Rasterizer:
    """One library context: workspace for up to `max_gaussians` Gaussians,
    `pair_capacity` Gaussian-tile pairs and images up to max_width x max_height."""

    def __init__(self, max_gaussians: int, pair_capacity: int, max_width: int, max_height: int,
                 device: int = 0):
        self.device = device
        self.ctx = _lib.adr_create(int(max_gaussians), int(pair_capacity), int(max_width),
                                   int(max_height), int(device))
        self.n = 0
        self.camera = None
        self.frame = 0          # increments per adr_preprocess; backward needs the last frame

    def close(self):
        if self.ctx:
            _lib.adr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stages -----------------------------------------------------------------
    def preprocess(self, params, camera, settings, stream=None):
        means, scales, rots, opac, sh = params
        n = check_params(params, self.device)
        self.n = n
        self.camera = camera
        self.frame += 1
        _lib.adr_preprocess(self.ctx, _ptr(means), _ptr(scales), _ptr(rots), _ptr(opac), _ptr(sh),
                            n, _lib.make_camera(camera), _lib.make_settings(settings),
                            _stream(stream))

    def sort(self, stream=None):
        _lib.adr_sort(self.ctx, _stream(stream))

    def render(self, img=None, t_final=None, load=None, stream=None, want_aux=True):
        h, w = self.camera.height, self.camera.width
        dev = f"cuda:{self.device}"
        if img is None:
            img = torch.empty((3, h, w), dtype=torch.float32, device=dev)
        if want_aux and t_final is None:
            t_final = torch.empty((h, w), dtype=torch.float32, device=dev)
        if want_aux and load is None:
            load = torch.empty((h, w), dtype=torch.int32, device=dev)
        check_tensor("img", img, 3 * h * w, device=self.device)
        if t_final is not None:
            check_tensor("t_final", t_final, h * w, device=self.device)
        if load is not None:
            check_tensor("load", load, h * w, dtype=torch.int32, device=self.device)
        _lib.adr_render(self.ctx, _ptr(img), _ptr(t_final), _ptr(load), _stream(stream))
        return img, t_final, load

    def forward(self, params, camera, settings, stream=None, **kw):
        self.preprocess(params, camera, settings, stream)
        self.sort(stream)
        return self.render(stream=stream, **kw)

    SLICES_NEVER, SLICES_ALWAYS, SLICES_ADAPTIVE = 0, 1, 2

    def set_tile_split(self, mode):
        """TILE_SPLIT_OFF (default) or TILE_SPLIT_LAST_SLICE: the last depth slice
        renders every unfinished tile as two half-tile CTAs (see adr.h)."""
        _lib.adr_set_tile_split(self.ctx, mode)

    def set_depth_slices(self, mode):
        """Depth slices of the frame: SLICES_NEVER, SLICES_ALWAYS or SLICES_ADAPTIVE
        (default); the images are the same, only the time differs."""
        _lib.adr_set_depth_slices(self.ctx, mode)

    def backward(self, params, dl_dimg, dl_dload=None, stream=None):
        """Gradients of the last rendered frame: (g_means, g_scales, g_rots, g_opac, g_sh)."""
        if check_params(params, self.device) != self.n:
            raise ValueError(f"backward needs the {self.n} Gaussians of the last frame")
        h, w = self.camera.height, self.camera.width
        grads = tuple(torch.empty_like(p) for p in params)
        dl_dimg = dl_dimg.contiguous().float()
        check_tensor("dl_dimg", dl_dimg, 3 * h * w, device=self.device)
        if dl_dload is not None:
            dl_dload = dl_dload.contiguous().float()
            check_tensor("dl_dload", dl_dload, h * w, device=self.device)
        _lib.adr_render_backward(self.ctx, *(_ptr(p) for p in params), _ptr(dl_dimg),
                                 _ptr(dl_dload), *(_ptr(g) for g in grads), _stream(stream))
        return grads

    def load_loss(self, load, weight=1.0, want_grad=True, stream=None):
        """(mean, std) of the per-pixel load and weight * dL_load/dl (Eq. 13)."""
        load = load.contiguous()
        check_tensor("load", load, load.numel(), dtype=torch.int32, device=self.device)
        stats = torch.empty(2, dtype=torch.float64, device=load.device)
        grad = torch.empty(load.shape, dtype=torch.float32, device=load.device) if want_grad else None
        _lib.adr_load_loss(self.ctx, _ptr(load), load.numel(), float(weight), _ptr(stats), _ptr(grad),
                           _stream(stream))
        return stats, grad

    # -- inspection -------------------------------------------------------------
    def num_pairs(self, raise_on_error=True):
        p, st = _lib.adr_num_pairs(self.ctx, raise_on_error)
        return (p, st) if not raise_on_error else p

    FRAME_COUNT_NAMES = ("pairs", "visible", "runs", "sliced", "runs_slice0", "runs_slice1",
                         "visible_slice1")

    def frame_counts(self):
        """Sizes of the last rendered frame (adr_frame_counts) as a dict."""
        buf = (ctypes.c_int64 * len(self.FRAME_COUNT_NAMES))()
        _lib.check(_lib.load().adr_frame_counts(self.ctx, ctypes.addressof(buf), len(buf)),
                   "adr_frame_counts")
        return dict(zip(self.FRAME_COUNT_NAMES, (int(v) for v in buf)))

    def read_pairs(self, count=None, stream=None):
        p = self.num_pairs() if count is None else count
        dev = f"cuda:{self.device}"
        keys = torch.empty(max(p, 1), dtype=torch.int64, device=dev)
        vals = torch.empty(max(p, 1), dtype=torch.int32, device=dev)
        _lib.adr_read_pairs(self.ctx, _ptr(keys), _ptr(vals), p, _stream(stream))
        torch.cuda.synchronize(self.device)
        return (keys[:p].cpu().numpy().view(np.uint64), vals[:p].cpu().numpy().view(np.uint32))

    def read_gaussians(self, stream=None):
        dev = f"cuda:{self.device}"
        n = max(self.n, 1)
        geom = torch.empty((n, _lib.ADR_GEOM_FLOATS), dtype=torch.float32, device=dev)
        rect = torch.empty((n, 4), dtype=torch.int32, device=dev)
        tiles = torch.empty((n,), dtype=torch.int32, device=dev)
        _lib.adr_read_gaussians(self.ctx, _ptr(geom), _ptr(rect), _ptr(tiles), _stream(stream))
        torch.cuda.synchronize(self.device)
        return (geom[:self.n].cpu().numpy(), rect[:self.n].cpu().numpy(),
                tiles[:self.n].cpu().numpy())

    def read_ranges(self, stream=None):
        cam = self.camera
        nt = ((cam.width + TILE - 1) // TILE) * ((cam.height + TILE - 1) // TILE)
        r = torch.empty((nt, 2), dtype=torch.int32, device=f"cuda:{self.device}")
        _lib.adr_read_ranges(self.ctx, _ptr(r), _stream(stream))
        torch.cuda.synchronize(self.device)
        return r.cpu().numpy().view(np.uint32)

    def read_pixel_stats(self, stream=None):
        h, w = self.camera.height, self.camera.width
        dev = f"cuda:{self.device}"
        last = torch.empty((h, w), dtype=torch.int32, device=dev)
        trav = torch.empty((h, w), dtype=torch.int32, device=dev)
        _lib.adr_read_pixel_stats(self.ctx, _ptr(last), _ptr(trav), _stream(stream))
        torch.cuda.synchronize(self.device)
        return last.cpu().numpy(), trav.cpu().numpy()

    def profile(self, enable: bool):
        _lib.adr_profile_enable(self.ctx, enable)

    def profile_read(self):
        return _lib.adr_profile_read(self.ctx)

    def trace_tiles(self, enable: bool):
        """Per-tile Render tracing on or off (adr_trace_tiles)."""
        _lib.check(_lib.load().adr_trace_tiles(self.ctx, 1 if enable else 0), "adr_trace_tiles")

    def read_tile_trace(self, stream=None):
        """The last frame's per-tile trace: uint32 numpy [2, tiles, 4] of
        (start ns, end ns, SM, staged positions) for slice 0 (or the whole
        list) and slice 1."""
        cam = self.camera
        nt = ((cam.width + TILE - 1) // TILE) * ((cam.height + TILE - 1) // TILE)
        out = torch.empty((2, nt, 4), dtype=torch.int32, device=f"cuda:{self.device}")
        _lib.check(_lib.load().adr_read_tile_trace(self.ctx, _ptr(out), _stream(stream)),
                   "adr_read_tile_trace")
        torch.cuda.synchronize(self.device)
        return out.cpu().numpy().view(np.uint32)

    def sync_status(self):
        return _lib.adr_sync_status(self.ctx)
