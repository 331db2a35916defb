"""ctypes binding of libadr.so — argument marshalling only.

Every function here has the name and argument order of its C counterpart in
include/adr.h.  Pointers are passed as integers (device addresses from
torch tensors' data_ptr(), or host addresses of numpy arrays); streams as
integers (torch.cuda.Stream.cuda_stream).  No computation happens here.
There is no fallback: if libadr.so cannot be loaded, the import fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ADR_OK = 0
ADR_ERR_INVALID = 1
ADR_ERR_CAPACITY = 2
ADR_ERR_CUDA = 3
ADR_ERR_TIMEOUT = 4
ADR_PENDING = 5
ADR_ERR_ADMISSION = 6
STATUS_NAMES = {0: "ADR_OK", 1: "ADR_ERR_INVALID", 2: "ADR_ERR_CAPACITY", 3: "ADR_ERR_CUDA",
                4: "ADR_ERR_TIMEOUT", 5: "ADR_PENDING", 6: "ADR_ERR_ADMISSION"}
ADR_TILE = 16
ADR_GEOM_FLOATS = 12


class AdrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class adr_camera(ctypes.Structure):
    _fields_ = [("view", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("near_z", ctypes.c_float),
                ("cam_pos", ctypes.c_float * 3), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class adr_settings(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("alpha_low", ctypes.c_float), ("t_min", ctypes.c_float),
                ("lowpass", ctypes.c_float), ("jac_clamp", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("sh_degree", ctypes.c_int32),
                ("rect_rule", ctypes.c_int32), ("load_grad", ctypes.c_int32)]


class adr_serve_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64),
                ("slot_pair_capacity", ctypes.c_int64), ("slot_max_gaussians", ctypes.c_int64),
                ("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_batch", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

# name -> (restype, argtypes)
_SIGNATURES = {
    "adr_create": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I32, _I32, _I32]),
    "adr_destroy": (None, [_P]),
    "adr_preprocess": (_I32, [_P, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(adr_camera),
                              ctypes.POINTER(adr_settings), _P]),
    "adr_sort": (_I32, [_P, _P]),
    "adr_render": (_I32, [_P, _P, _P, _P, _P]),
    "adr_num_pairs": (_I32, [_P, ctypes.POINTER(_I64)]),
    "adr_frame_counts": (_I32, [_P, _P, _I32]),
    "adr_read_pairs": (_I32, [_P, _P, _P, _I64, _P]),
    "adr_read_gaussians": (_I32, [_P, _P, _P, _P, _P]),
    "adr_read_ranges": (_I32, [_P, _P, _P]),
    "adr_sync_status": (_I32, [_P]),
    "adr_test_lookback_expiry": (_I32, [_I32, _I32]),
    "adr_read_pixel_stats": (_I32, [_P, _P, _P, _P]),
    "adr_render_host": (_I32, [_P, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(adr_camera),
                               ctypes.POINTER(adr_settings), _P, _P, _P, _P]),
    "adr_render_frame_noalloc": (_I32, [_P, _P, _P, _P, _P, _I64, ctypes.POINTER(adr_camera),
                                        ctypes.POINTER(adr_settings), _P, _P, _P, _P]),
    "adr_render_backward": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "adr_load_loss": (_I32, [_P, _P, _I64, ctypes.c_float, _P, _P, _P]),
    "adr_image_loss": (_I32, [_P, _P, _I32, _I32, _I32, ctypes.c_float, ctypes.c_float, _P, _P,
                              _P, _P]),
    "adr_profile_enable": (_I32, [_P, _I32]),
    "adr_set_depth_slices": (_I32, [_P, _I32]),
    "adr_set_host_reads": (_I32, [_P, _I32]),
    "adr_set_tile_split": (_I32, [_P, _I32]),
    "adr_profile_read": (_I32, [_P, _I32, _P, _P, _P, ctypes.POINTER(_I32)]),
    "adr_profile_kernel_name": (ctypes.c_char_p, [_I32]),
    "adr_trace_tiles": (_I32, [_P, _I32]),
    "adr_read_tile_trace": (_I32, [_P, _P, _P]),
    "adr_serve_create": (_I32, [ctypes.POINTER(_P), ctypes.POINTER(adr_serve_config)]),
    "adr_serve_destroy": (None, [_P]),
    "adr_serve_add_scene": (_I32, [_P, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(adr_settings),
                                   ctypes.POINTER(_I32)]),
    "adr_serve_submit": (_I32, [_P, _I32, ctypes.POINTER(adr_camera), _P,
                                ctypes.POINTER(ctypes.c_uint64)]),
    "adr_serve_poll": (_I32, [_P, ctypes.c_uint64, _I64]),
    "adr_serve_stats": (_I32, [_P, _P, _I32]),
    "adr_serve_reset_stats": (_I32, [_P]),
    "adr_last_error": (ctypes.c_char_p, []),
    "adr_version": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libadr.so (building it first if asked and it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libadr.so not found at {path}; run __graft_entry__.build()")
            import torch  # noqa: F401  (load torch's libcudart first so one runtime is shared)
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_names():
    return list(_SIGNATURES)


def last_error() -> str:
    return load().adr_last_error().decode()


def check(status: int, what: str = "") -> int:
    if status != ADR_OK and status != ADR_PENDING:
        raise AdrError(status, f"{what}: {last_error()}")
    return status


def make_camera(cam) -> adr_camera:
    """Build the C struct from a scenes.Camera."""
    c = adr_camera()
    v = cam.view.reshape(-1)
    for i in range(16):
        c.view[i] = float(v[i])
    c.fx, c.fy, c.cx, c.cy, c.near_z = cam.fx, cam.fy, cam.cx, cam.cy, cam.near
    for i in range(3):
        c.cam_pos[i] = float(cam.cam_pos[i])
    c.width, c.height = cam.width, cam.height
    return c


def make_settings(st) -> adr_settings:
    s = adr_settings()
    s.mode = int(st.mode)
    s.alpha_low, s.t_min, s.lowpass, s.jac_clamp = st.alpha_low, st.t_min, st.lowpass, st.jac_clamp
    for i in range(3):
        s.bg[i] = float(st.bg[i])
    s.sh_degree = int(st.sh_degree)
    s.rect_rule = int(st.rect_rule)
    s.load_grad = int(st.load_grad)
    return s


# Thin call-throughs with the C names (pointers as ints).
def adr_create(max_gaussians, pair_capacity, max_width, max_height, device=0):
    out = _P()
    check(load().adr_create(ctypes.byref(out), max_gaussians, pair_capacity, max_width,
                            max_height, device), "adr_create")
    return out.value


def adr_destroy(ctx):
    load().adr_destroy(ctx)


def adr_preprocess(ctx, means, scales, rots, opac, sh, n, camera, settings, stream):
    return check(load().adr_preprocess(ctx, means, scales, rots, opac, sh, n,
                                       ctypes.byref(camera), ctypes.byref(settings), stream),
                 "adr_preprocess")


def adr_sort(ctx, stream):
    return check(load().adr_sort(ctx, stream), "adr_sort")


def adr_render(ctx, img, t_final, load_, stream):
    return check(load().adr_render(ctx, img, t_final, load_, stream), "adr_render")


def adr_num_pairs(ctx, raise_on_error=True):
    p = _I64(0)
    st = load().adr_num_pairs(ctx, ctypes.byref(p))
    if raise_on_error:
        check(st, "adr_num_pairs")
    return p.value, st


def adr_read_pairs(ctx, keys, vals, capacity, stream):
    return check(load().adr_read_pairs(ctx, keys, vals, capacity, stream), "adr_read_pairs")


def adr_read_gaussians(ctx, geom, rect, tiles, stream):
    return check(load().adr_read_gaussians(ctx, geom, rect, tiles, stream), "adr_read_gaussians")


def adr_read_ranges(ctx, ranges, stream):
    return check(load().adr_read_ranges(ctx, ranges, stream), "adr_read_ranges")


def adr_read_pixel_stats(ctx, last, traversed, stream):
    return check(load().adr_read_pixel_stats(ctx, last, traversed, stream), "adr_read_pixel_stats")


def adr_sync_status(ctx):
    return load().adr_sync_status(ctx)


def adr_test_lookback_expiry(withheld_chunk, spin_limit=64):
    """Testing hook: make the run scan's lookback waits give up (see adr.h)."""
    return load().adr_test_lookback_expiry(int(withheld_chunk), int(spin_limit))


def adr_render_host(ctx, means, scales, rots, opac, sh, n, camera, settings, img, t_final, load_,
                    stream):
    return check(load().adr_render_host(ctx, means, scales, rots, opac, sh, n,
                                        ctypes.byref(camera), ctypes.byref(settings), img,
                                        t_final, load_, stream), "adr_render_host")


def adr_render_backward(ctx, means, scales, rots, opac, sh, dl_dimg, dl_dload, g_means, g_scales,
                        g_rots, g_opac, g_sh, stream):
    return check(load().adr_render_backward(ctx, means, scales, rots, opac, sh, dl_dimg, dl_dload,
                                            g_means, g_scales, g_rots, g_opac, g_sh, stream),
                 "adr_render_backward")


def adr_load_loss(ctx, load_, hw, weight, stats, dl_dload, stream):
    return check(load().adr_load_loss(ctx, load_, hw, weight, stats, dl_dload, stream),
                 "adr_load_loss")


def adr_image_loss(img, ref, channels, height, width, w_l1, w_ssim, stats, dl_dimg, scratch,
                   stream):
    return check(load().adr_image_loss(img, ref, channels, height, width, w_l1, w_ssim, stats,
                                       dl_dimg, scratch, stream), "adr_image_loss")


def adr_set_depth_slices(ctx, mode):
    return check(load().adr_set_depth_slices(ctx, int(mode)), "adr_set_depth_slices")


HOST_READ_COPY, HOST_READ_MAPPED = 0, 1


def adr_set_host_reads(ctx, mode):
    return check(load().adr_set_host_reads(ctx, int(mode)), "adr_set_host_reads")


TILE_SPLIT_OFF, TILE_SPLIT_LAST_SLICE = 0, 1


def adr_set_tile_split(ctx, mode):
    return check(load().adr_set_tile_split(ctx, int(mode)), "adr_set_tile_split")


def adr_profile_enable(ctx, enable):
    return check(load().adr_profile_enable(ctx, 1 if enable else 0), "adr_profile_enable")


def adr_profile_read(ctx, max_kernels=16):
    """{kernel name: (total ms, launches)} since the last read."""
    import numpy as np
    ids = np.zeros(max_kernels, np.int32)
    ms = np.zeros(max_kernels, np.float64)
    cnt = np.zeros(max_kernels, np.int32)
    k = _I32(0)
    check(load().adr_profile_read(ctx, max_kernels, ids.ctypes.data, ms.ctypes.data,
                                  cnt.ctypes.data, ctypes.byref(k)), "adr_profile_read")
    lib = load()
    return {lib.adr_profile_kernel_name(int(ids[i])).decode(): (float(ms[i]), int(cnt[i]))
            for i in range(k.value)}


def adr_version():
    return load().adr_version().decode()
