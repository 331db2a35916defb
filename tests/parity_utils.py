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


def compare_images(img, t_final, load, ref, exclude, atol=1e-4):
    """Max abs error per channel within atol on every pixel not excluded.
    Returns (max error, number of excluded pixels)."""
    keep = ~exclude
    err = np.abs(img.astype(np.float64) - ref["img"])
    worst = float(err[:, keep].max()) if keep.any() else 0.0
    if worst > atol:
        c, y, x = np.unravel_index(np.argmax(np.where(keep[None], err, 0)), err.shape)
        raise AssertionError(f"image error {worst:.3e} > {atol} at channel {c} pixel ({x},{y}): "
                             f"gpu {img[c, y, x]!r} oracle {ref['img'][c, y, x]!r}")
    terr = np.abs(t_final.astype(np.float64) - ref["t_final"])[keep]
    assert terr.size == 0 or terr.max() <= atol, f"t_final error {terr.max():.3e}"
    # the per-pixel load is an integer decision: exact except at excluded pixels
    lbad = np.count_nonzero((load != ref["load"]) & keep)
    assert lbad == 0, f"{lbad} pixels with a different load l_i"
    return worst, int(exclude.sum())
