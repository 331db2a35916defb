"""Python face of the serving scheduler (adr_serve_* in include/adr.h):
argument marshalling only; scheduling, admission and rendering run in
libadr.so."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .raster import check_params, check_tensor

STAT_NAMES = ("completed", "p50_ms", "p99_ms", "mean_ms", "max_inflight", "admitted_while_busy",
              "rejected", "frames_per_s", "capacity_errors", "graph_replays", "batches",
              "largest_batch", "mean_batch")


class Server:
    """Resident scenes + a continuous-batching render loop on one device."""

    def __init__(self, max_slots=4, mem_budget_bytes=8 << 30, slot_pair_capacity=1 << 27,
                 slot_max_gaussians=1 << 22, max_width=1920, max_height=1080, use_graphs=True,
                 device=None, max_batch=1):
        self._lib = _lib.load()
        dev = torch.cuda.current_device() if device is None else int(device)
        cfg = _lib.adr_serve_config(max_slots=max_slots, mem_budget_bytes=int(mem_budget_bytes),
                                    slot_pair_capacity=int(slot_pair_capacity),
                                    slot_max_gaussians=int(slot_max_gaussians),
                                    max_width=max_width, max_height=max_height,
                                    use_graphs=1 if use_graphs else 0, device=dev,
                                    max_batch=int(max_batch))
        h = ctypes.c_void_p()
        _lib.check(self._lib.adr_serve_create(ctypes.byref(h), ctypes.byref(cfg)), "adr_serve_create")
        self._h = h
        self.device = dev
        self._scenes = []   # keep the borrowed tensors alive

    def _check_out(self, camera, out):
        """The request's image [3, H, W] is written in full by the device."""
        if not isinstance(out, torch.Tensor) or tuple(out.shape) != (3, camera.height, camera.width):
            raise ValueError(f"out must be a [3, {camera.height}, {camera.width}] tensor")
        check_tensor("out", out, 3 * camera.height * camera.width, device=self.device)

    def add_scene(self, params, settings) -> int:
        n = check_params(params, self.device)
        means, scales, rots, opac, sh = params
        sid = ctypes.c_int32()
        st = _lib.make_settings(settings)
        _lib.check(self._lib.adr_serve_add_scene(self._h, means.data_ptr(), scales.data_ptr(),
                                                 rots.data_ptr(), opac.data_ptr(), sh.data_ptr(),
                                                 n, ctypes.byref(st), ctypes.byref(sid)),
                   "adr_serve_add_scene")
        self._scenes.append(params)
        return sid.value

    def submit(self, scene_id: int, camera, out: torch.Tensor) -> int:
        self._check_out(camera, out)
        c = _lib.make_camera(camera)
        t = ctypes.c_uint64()
        _lib.check(self._lib.adr_serve_submit(self._h, scene_id, ctypes.byref(c), out.data_ptr(),
                                              ctypes.byref(t)), "adr_serve_submit")
        return t.value

    def submit_status(self, scene_id: int, camera, out: torch.Tensor) -> int:
        """Like submit but returns the raw status (no exception from the library)."""
        self._check_out(camera, out)
        c = _lib.make_camera(camera)
        t = ctypes.c_uint64()
        return self._lib.adr_serve_submit(self._h, scene_id, ctypes.byref(c), out.data_ptr(),
                                          ctypes.byref(t))

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        """Raw status: ADR_OK, ADR_PENDING, ADR_ERR_TIMEOUT or a request error.
        A negative timeout waits for an hour."""
        return self._lib.adr_serve_poll(self._h, ticket, 3_600_000_000 if timeout_us < 0 else timeout_us)

    def wait(self, ticket: int):
        _lib.check(self.poll(ticket), "adr_serve_poll")

    def stats(self) -> dict:
        buf = (ctypes.c_double * len(STAT_NAMES))()
        _lib.check(self._lib.adr_serve_stats(self._h, ctypes.addressof(buf), len(STAT_NAMES)),
                   "adr_serve_stats")
        return dict(zip(STAT_NAMES, list(buf)))

    def reset_stats(self):
        _lib.check(self._lib.adr_serve_reset_stats(self._h), "adr_serve_reset_stats")

    def close(self):
        if self._h:
            self._lib.adr_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
