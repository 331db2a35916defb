"""CPU oracle for the AdR-Gaussian rasterization path — TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package.  The product library never loads it; it shares no
code with the CUDA sources.  `adr_oracle.c` (FP64 C) holds the forward path;
`grad.py` holds the FP64 PyTorch restatement used for analytic gradients.

Each wrapper below mirrors one C function and cites the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16
GEOM = 16
G_PX, G_PY, G_COV_A, G_COV_B, G_COV_C, G_CONIC_A, G_CONIC_B, G_CONIC_C, \
    G_LAMBDA, G_RO, G_RX, G_RY, G_VX, G_VY, G_VZ, G_OPAC = range(16)
F_VISIBLE = 1
F_NEAR = 2


def compile_library(src: str, out: str) -> str:
    """gcc a C source of the oracle into a shared library (IEEE double, no FMA
    contraction).  The tests also compile deliberately broken copies with it."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile adr_oracle.c (when the library is missing or older than it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_library(_SRC, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """Open a compiled oracle and declare its functions' signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_preprocess.restype = i64
    lib.orc_preprocess.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, i32, i32, dbl, dbl, dbl,
                                   dbl, P, P, P, P, P, P]
    lib.orc_emit_pairs.restype = i64
    lib.orc_emit_pairs.argtypes = [i64, P, P, P, i32, P, P, i64]
    lib.orc_sort_pairs.restype = None
    lib.orc_sort_pairs.argtypes = [i64, P, P]
    lib.orc_tile_ranges.restype = None
    lib.orc_tile_ranges.argtypes = [i64, P, i32, P]
    lib.orc_render_tiled.restype = None
    lib.orc_render_tiled.argtypes = [i32, i32, P, P, P, P, dbl, dbl, P, dbl, dbl,
                                     P, P, P, P, P, P]
    lib.orc_render_brute.restype = None
    lib.orc_render_brute.argtypes = [i64, i32, i32, P, P, P, P, P, dbl, dbl, P, P, P, P]
    lib.orc_load_std.restype = dbl
    lib.orc_load_std.argtypes = [i64, P]
    lib.orc_real_sh.restype = dbl
    lib.orc_real_sh.argtypes = [i32, i32, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def real_sh(l: int, m: int, d) -> float:
    """Real spherical harmonic Y_{l,m}(d), Condon-Shortley phase (colour model, Sec. 3.1)."""
    d = _c(d, np.float64)
    return _load().orc_real_sh(l, m, _p(d))


def preprocess(scene, camera, settings, tol_rel: float = 1e-6):
    """Stage 1, Preprocess, with the adaptive-radius (Eq. 7-8) or AABB (Eq. 10-11)
    early cull selected by `settings.mode`.  Returns a dict of per-Gaussian arrays."""
    lib = _load()
    n = scene.n
    # float32 inputs promote exactly; float64 inputs (finite differences) pass through
    means, scales, rots, opac, sh = (_c(a, np.float64) for a in scene.arrays())
    cam = _c(camera.record(), np.float32)
    geom = np.zeros((n, GEOM), np.float64)
    depth = np.zeros(n, np.float32)
    rect = np.zeros((n, 4), np.int32)
    tiles = np.zeros(n, np.int64)
    rgb = np.zeros((n, 3), np.float64)
    flags = np.zeros(n, np.uint8)
    total = lib.orc_preprocess(n, _p(means), _p(scales), _p(rots), _p(opac), _p(sh),
                               settings.sh_degree, _p(cam), camera.width, camera.height,
                               settings.mode, settings.rect_rule,
                               settings.alpha_low, settings.lowpass,
                               settings.jac_clamp, tol_rel, _p(geom), _p(depth), _p(rect),
                               _p(tiles), _p(rgb), _p(flags))
    return dict(geom=geom, depth=depth, rect=rect, tiles=tiles, rgb=rgb, flags=flags,
                num_pairs=int(total), width=camera.width, height=camera.height)


def emit_pairs(pre):
    """Stages 2-3: exclusive scan of tile counts and key emission
    key = (tile << 32) | bits(depth), value = Gaussian index (Sec. 3.2)."""
    lib = _load()
    n = pre["tiles"].shape[0]
    p = pre["num_pairs"]
    keys = np.zeros(max(p, 1), np.uint64)
    vals = np.zeros(max(p, 1), np.uint32)
    got = lib.orc_emit_pairs(n, _p(pre["rect"]), _p(pre["tiles"]), _p(pre["depth"]),
                             pre["width"], _p(keys), _p(vals), p)
    assert got == p
    return keys[:p], vals[:p]


def sort_pairs(keys, vals):
    """Stage 4: stable ascending sort by key (tile, then depth)."""
    keys = keys.copy()
    vals = vals.copy()
    _load().orc_sort_pairs(keys.shape[0], _p(keys), _p(vals))
    return keys, vals


def tile_ranges(keys, width, height):
    """Stage 5: [start, end) of each tile's run in the sorted list."""
    tx = (width + TILE - 1) // TILE
    ty = (height + TILE - 1) // TILE
    ranges = np.zeros((tx * ty, 2), np.uint32)
    _load().orc_tile_ranges(keys.shape[0], _p(_c(keys, np.uint64)), tx * ty, _p(ranges))
    return ranges


def render_tiled(pre, ranges, vals, settings, tol_alpha=1e-4, tol_t=1e-4):
    """Stage 6: per-pixel front-to-back blending over the tile's sorted list
    (Eq. 2-3) with the per-pixel load l_i (Eq. 12)."""
    w, h = pre["width"], pre["height"]
    img = np.zeros((3, h, w), np.float64)
    t_final = np.zeros((h, w), np.float64)
    load = np.zeros((h, w), np.int32)
    last = np.zeros((h, w), np.int32)
    trav = np.zeros((h, w), np.int32)
    near = np.zeros((h, w), np.uint8)
    bg = _c(settings.bg, np.float64)
    vals = _c(vals, np.uint32)
    if vals.size == 0:
        vals = np.zeros(1, np.uint32)
    _load().orc_render_tiled(w, h, _p(_c(ranges, np.uint32)), _p(vals), _p(pre["geom"]),
                             _p(pre["rgb"]), settings.alpha_low, settings.t_min, _p(bg),
                             tol_alpha, tol_t, _p(img), _p(t_final), _p(load), _p(last),
                             _p(trav), _p(near))
    return dict(img=img, t_final=t_final, load=load, last=last, traversed=trav, near=near)


def render_brute(pre, settings, use_rect: bool = False):
    """Eq. 2-3 per pixel over every visible Gaussian in (depth, index) order,
    with no tiles; with `use_rect` a Gaussian only reaches pixels of its tiles."""
    w, h = pre["width"], pre["height"]
    n = pre["tiles"].shape[0]
    img = np.zeros((3, h, w), np.float64)
    t_final = np.zeros((h, w), np.float64)
    load = np.zeros((h, w), np.int32)
    bg = _c(settings.bg, np.float64)
    rect = _p(pre["rect"]) if use_rect else None
    _load().orc_render_brute(n, w, h, _p(pre["flags"]), _p(pre["depth"]), rect, _p(pre["geom"]),
                             _p(pre["rgb"]), settings.alpha_low, settings.t_min, _p(bg),
                             _p(img), _p(t_final), _p(load))
    return dict(img=img, t_final=t_final, load=load)


def load_std(load) -> float:
    """L_load = std over pixels of l_i (Eq. 13)."""
    load = _c(load, np.int32).reshape(-1)
    return _load().orc_load_std(load.shape[0], _p(load))


def render(scene, camera, settings, tol_rel=1e-6, tol_alpha=1e-4, tol_t=1e-4):
    """The whole forward path: preprocess, pairs, sort, ranges, tiled render."""
    pre = preprocess(scene, camera, settings, tol_rel)
    keys, vals = emit_pairs(pre)
    skeys, svals = sort_pairs(keys, vals)
    ranges = tile_ranges(skeys, camera.width, camera.height)
    out = render_tiled(pre, ranges, svals, settings, tol_alpha, tol_t)
    out.update(pre=pre, keys=skeys, vals=svals, ranges=ranges)
    return out
