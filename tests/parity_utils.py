"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs and compare them."""
from __future__ import annotations

import numpy as np

import oracle

TILE = 16


def gpu_forward(rast, params, cam, st):
    import torch
    img, t_final, load = rast.forward(params, cam, st)
    torch.cuda.synchronize()
    return img.cpu().numpy(), t_final.cpu().numpy(), load.cpu().numpy()


def pair_tiles_by_gaussian(keys, vals):
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    out = {}
    for t, g in zip(tiles.tolist(), vals.tolist()):
        out.setdefault(g, set()).add(t)
    return out


def compare_pairs(gpu_keys, gpu_vals, orc_keys, orc_vals, orc_flags):
    """Sorted pair lists must be bit-exact once the pairs of Gaussians whose
    cull or tile decision lies within tolerance of its threshold (oracle flag
    F_NEAR) are set aside.  Returns (near Gaussians whose tiles differ, the
    set of tiles those differences touch)."""
    near = (orc_flags & oracle.F_NEAR) != 0
    gm = ~near[gpu_vals.astype(np.int64)] if gpu_vals.size else np.zeros(0, bool)
    om = ~near[orc_vals.astype(np.int64)] if orc_vals.size else np.zeros(0, bool)
    gk, gv = gpu_keys[gm], gpu_vals[gm]
    ok_, ov = orc_keys[om], orc_vals[om]
    assert gk.shape == ok_.shape, f"pair count differs: gpu {gk.shape[0]} vs oracle {ok_.shape[0]}"
    bad = np.nonzero((gk != ok_) | (gv != ov))[0]
    assert bad.size == 0, (f"{bad.size} pairs differ; first at {bad[0]}: gpu ({gk[bad[0]]:#x}, "
                           f"{gv[bad[0]]}) oracle ({ok_[bad[0]]:#x}, {ov[bad[0]]})")
    # near Gaussians: log differences
    g_near = pair_tiles_by_gaussian(gpu_keys[~gm], gpu_vals[~gm])
    o_near = pair_tiles_by_gaussian(orc_keys[~om], orc_vals[~om])
    differing, tiles = [], set()
    for g in set(g_near) | set(o_near):
        a, b = g_near.get(g, set()), o_near.get(g, set())
        if a != b:
            differing.append(g)
            tiles |= a ^ b
    return differing, tiles


def tile_mask(tiles, width, height):
    m = np.zeros((height, width), bool)
    tx = (width + TILE - 1) // TILE
    for t in tiles:
        y0, x0 = (t // tx) * TILE, (t % tx) * TILE
        m[y0:y0 + TILE, x0:x0 + TILE] = True
    return m


def compare_images(img, t_final, load, ref, exclude, atol=1e-4, max_logged_frac=1e-4):
    """Every pixel where the GPU and the oracle disagree (any channel or the
    final transmittance off by more than atol, or a different load l_i) must
    be an excluded (near-threshold) pixel, and the number of such logged
    pixels must stay within max_logged_frac of the image.
    Returns (max error over kept pixels, logged pixels, excluded pixels)."""
    err = np.abs(img.astype(np.float64) - ref["img"]).max(axis=0)
    terr = np.abs(t_final.astype(np.float64) - ref["t_final"])
    mism = (err > atol) | (terr > atol) | (load != ref["load"])
    bad = mism & ~exclude
    if bad.any():
        y, x = np.argwhere(bad)[0]
        raise AssertionError(
            f"{int(bad.sum())} non-excluded pixels differ; first ({x},{y}): gpu "
            f"{img[:, y, x]} T={t_final[y, x]} l={load[y, x]} oracle {ref['img'][:, y, x]} "
            f"T={ref['t_final'][y, x]} l={ref['load'][y, x]}")
    logged = int(mism.sum())
    hw = img.shape[1] * img.shape[2]
    assert logged <= max(4, max_logged_frac * hw), f"{logged} near-threshold pixels differ"
    keep = ~exclude
    worst = float(err[keep].max()) if keep.any() else 0.0
    return worst, logged, int(exclude.sum())
