"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bar (from the target): Gaussian-tile pairs and sorted keys bit-exact, except
pairs whose cull/tile decision lies within 1e-6 (relative) of its threshold,
which are logged; images within 1e-4 max abs per channel, excluding pixels
whose blend decisions lie within tolerance of a threshold in the FP64
oracle (alpha vs alpha_low within 1e-4 relative: in FP32 the minor-axis
offset of a pixel from a long, thin Gaussian is off by ~1e-7 times its
distance along the major axis, which at the workloads' largest Gaussians
moves alpha by up to ~1e-4; T(1-alpha) vs t_min within 1e-4 — after a
few blends of alpha ~0.9 the FP32 transmittance carries ~1e-5 relative
error, so the stop decision gets the wider band) and the tiles
touched by logged pairs.  Every pixel that actually differs must be flagged,
and at most 1e-4 of the pixels may differ.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_08669_gb300 import scenes as S
from parity_utils import compare_images, compare_pairs, gpu_forward, tile_mask

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rast():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300.raster import Rasterizer
    r = Rasterizer(max_gaussians=1 << 20, pair_capacity=1 << 24, max_width=2048, max_height=2048)
    yield r
    r.close()


def _check_frame(rast, scene, cam, st, label=""):
    from paper_2409_08669_gb300.raster import upload
    params = upload(scene)
    img, t_final, load = gpu_forward(rast, params, cam, st)
    ref = oracle.render(scene, cam, st)
    pre = ref["pre"]
    flags = pre["flags"]
    near = (flags & oracle.F_NEAR) != 0
    geom, rect, tiles = rast.read_gaussians()
    # depth sort keys: bit-exact for every Gaussian (a NaN depth, whose payload
    # bits are not fixed, only has to be NaN on both sides)
    gd, od = geom[:, 11], pre["depth"]
    np.testing.assert_array_equal(np.isnan(gd), np.isnan(od))
    fin = ~np.isnan(od)
    np.testing.assert_array_equal(gd[fin].view(np.uint32), od[fin].view(np.uint32))
    # tile counts and rectangles: exact except near-threshold Gaussians
    tbad = np.nonzero((tiles != pre["tiles"]) & ~near)[0]
    assert tbad.size == 0, f"{label}: {tbad.size} Gaussians with different tile counts, e.g. {tbad[:5]}"
    has = tiles > 0
    rbad = np.nonzero(np.any(rect != pre["rect"], axis=1) & has & ~near)[0]
    assert rbad.size == 0, f"{label}: rect differs for {rbad[:5]}"
    # continuous per-Gaussian values where the Gaussian has pairs
    g = pre["geom"]
    np.testing.assert_allclose(geom[has, 0], g[has, oracle.G_PX], rtol=0, atol=2e-4)
    np.testing.assert_allclose(geom[has, 1], g[has, oracle.G_PY], rtol=0, atol=2e-4)
    np.testing.assert_allclose(geom[has, 8:11], pre["rgb"][has], rtol=2e-5, atol=2e-6)
    np.testing.assert_allclose(geom[has, 5], g[has, oracle.G_OPAC], rtol=0, atol=0)
    # sorted pairs
    keys, vals = rast.read_pairs()
    differing, dtiles = compare_pairs(keys, vals, ref["keys"], ref["vals"], flags)
    if not differing:
        ranges = rast.read_ranges()
        np.testing.assert_array_equal(ranges, ref["ranges"])
    exclude = (ref["near"] != 0) | tile_mask(dtiles, cam.width, cam.height)
    worst, logged, n_ex = compare_images(img, t_final, load, ref, exclude)
    hw = cam.width * cam.height
    print(f"{label}: P={keys.size} near-Gaussians={int(near.sum())} differing={len(differing)} "
          f"max|err|={worst:.2e} logged={logged} flagged={n_ex}/{hw}")
    return img, load


@pytest.mark.parametrize("mode", [S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB])
def test_tiny_scene_parity(rast, mode):
    """10k Gaussians, 256x256, one camera at distance 3 (the small workload)."""
    scene = S.tiny_scene(0)
    cam = S.look_at((0, 0, -3), width=256, height=256)
    _check_frame(rast, scene, cam, S.Settings(mode=mode), f"tiny/{S.MODE_NAMES[mode]}")


def test_ragged_image_many_tiles(rast):
    scene = S.tiny_scene(11, n=6000)
    cam = S.look_at((0.3, -0.2, -2.2), width=250, height=190)
    for mode in (S.MODE_PLAIN, S.MODE_AABB):
        _check_frame(rast, scene, cam, S.Settings(mode=mode), f"ragged/{mode}")


@pytest.mark.parametrize("mode", [S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB])
def test_3dgs_rect_rule_parity(rast, mode):
    """The 3DGS-compatible tile rounding, on the ragged image (250x190)."""
    scene = S.tiny_scene(11, n=6000)
    cam = S.look_at((0.3, -0.2, -2.2), width=250, height=190)
    st = S.Settings(mode=mode, rect_rule=S.RECT_3DGS)
    _check_frame(rast, scene, cam, st, f"rect3dgs/{S.MODE_NAMES[mode]}")


def test_wide_depth_span_sort_parity(rast):
    """Visible depths over 17 octaves (depth keys spanning more than 2^27, so
    every byte of the key varies and all four depth passes reorder); pairs
    and image against the oracle."""
    scene = S.deep_scene()
    cam = S.look_at((0, 0, -3), width=320, height=240)
    ref = oracle.render(scene, cam, S.Settings(mode=S.MODE_AABB))
    keys = ref["pre"]["depth"][ref["pre"]["tiles"] > 0].astype(np.float32).view(np.uint32)
    assert int(keys.max()) - (int(keys.min()) & ~511) >= 1 << 27
    _check_frame(rast, scene, cam, S.Settings(mode=S.MODE_AABB), "deep/aabb")


def test_cluster_scene_1080p_subset(rast):
    """A 200k-Gaussian draw of the clustered scene at 1920x1080 (tile grid 120x68)."""
    scene = S.cluster_scene(n=200_000, seed=1)
    cam = S.orbit_cameras(50, width=1920, height=1080)[7]
    _check_frame(rast, scene, cam, S.Settings(mode=S.MODE_AABB), "cluster1080")


# The alpha_low sweep (raising the splatting-opacity threshold above 1/255
# trades a little accuracy for speed, Sec. 5.4.1): the cull radii (Eq. 7,
# Eq. 10) and the per-pixel skip both move with alpha_low, and the oracle
# takes the same setting.
ALPHA_LOWS = [float(np.float32(2.0 / 255.0)), float(np.float32(4.0 / 255.0))]


@pytest.mark.parametrize("alpha_low", ALPHA_LOWS, ids=["2/255", "4/255"])
@pytest.mark.parametrize("mode", [S.MODE_PLAIN, S.MODE_AABB])
def test_alpha_low_sweep_tiny_parity(rast, mode, alpha_low):
    scene = S.tiny_scene(0)
    cam = S.look_at((0, 0, -3), width=256, height=256)
    st = S.Settings(mode=mode, alpha_low=alpha_low)
    _check_frame(rast, scene, cam, st, f"tiny/{S.MODE_NAMES[mode]}/alpha_low={alpha_low:.5f}")


@pytest.mark.parametrize("alpha_low", ALPHA_LOWS, ids=["2/255", "4/255"])
@pytest.mark.parametrize("mode", [S.MODE_PLAIN, S.MODE_AABB])
def test_alpha_low_sweep_cluster_1080p_parity(rast, mode, alpha_low):
    scene = S.cluster_scene(n=200_000, seed=1)
    cam = S.orbit_cameras(50, width=1920, height=1080)[7]
    st = S.Settings(mode=mode, alpha_low=alpha_low)
    _check_frame(rast, scene, cam, st, f"cluster1080/{S.MODE_NAMES[mode]}/alpha_low={alpha_low:.5f}")


def test_modes_render_identical_images_on_gpu(rast):
    """Losslessness (Sec. 5.2-5.3): culling changes no pixel."""
    from paper_2409_08669_gb300.raster import upload
    scene = S.cluster_scene(n=100_000, seed=5)
    cam = S.orbit_cameras(50, width=1280, height=720)[3]
    params = upload(scene)
    out = {}
    pairs = {}
    for mode in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB):
        img, t, load = gpu_forward(rast, params, cam, S.Settings(mode=mode))
        out[mode] = (img, t, load)
        pairs[mode] = rast.num_pairs()
    ref = oracle.render(scene, cam, S.Settings(mode=S.MODE_AABB))
    near = ref["near"] != 0
    for mode in (S.MODE_CIRCLE, S.MODE_AABB):
        diff = np.any(out[mode][0] != out[S.MODE_PLAIN][0], axis=0)
        assert np.count_nonzero(diff & ~near) == 0
        assert np.array_equal(out[mode][2][~near], out[S.MODE_PLAIN][2][~near])
    assert pairs[S.MODE_AABB] < pairs[S.MODE_CIRCLE] < pairs[S.MODE_PLAIN]


@pytest.mark.parametrize("theta,op", [(0.4, 0.3), (1.0, 0.95)])
def test_single_gaussian_footprint_closed_form(rast, theta, op):
    """One Gaussian at the image centre: image = c * min(0.99, sigma e^{-q/2})
    on the alpha >= 1/255 footprint (within the r_o tiles), 0 elsewhere."""
    from paper_2409_08669_gb300.raster import upload
    z0, s1, s2 = 3.0, 0.04, 0.015
    w, h = 96, 80
    cam = S.look_at((0, 0, -z0), width=w, height=h)
    dc = (0.9, 0.2, 0.5)
    q = (math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2))
    scene = S.isolated_gaussian((0, 0, 0), (s1, s2, 0.01), q, op, dc)
    img, t_final, load = gpu_forward(rast, upload(scene), cam, S.Settings())
    ref = oracle.render(scene, cam, S.Settings())
    # the oracle is pinned to the closed form on the same case (test_oracle_pins)
    np.testing.assert_allclose(img, ref["img"], atol=2e-6)
    assert ref["near"].sum() == 0
    np.testing.assert_array_equal(load[ref["near"] == 0], ref["load"][ref["near"] == 0])


def test_opaque_stack_with_zero_t_min_counts_every_blend(rast):
    """t_min = 0 (no early termination): behind a few dozen Gaussians of alpha
    near 0.99 the FP32 transmittance of the central pixels underflows to 0, yet every
    later Gaussian that reaches alpha_low there is still blended (with zero
    weight) and counted in l_i (Eq. 12), as in the FP64 oracle, where T never
    reaches 0."""
    from paper_2409_08669_gb300.raster import upload
    k = 100
    means = np.zeros((k, 3))
    means[:, 2] = np.linspace(0.0, 1.2, k)
    rgb = np.stack([np.linspace(0.1, 0.9, k), np.full(k, 0.5), np.linspace(0.9, 0.1, k)], axis=1)
    sh = np.zeros((k, 16, 3))
    sh[:, 0, :] = (rgb - 0.5) / 0.28209479177387814   # DC band: colour = Y00 * c + 0.5
    scene = S._pack(means, np.tile([0.2, 0.15, 0.01], (k, 1)), np.tile([1.0, 0.0, 0.0, 0.0], (k, 1)),
                    np.full(k, 0.995), sh)
    cam = S.look_at((0, 0, -3), width=64, height=48)
    st = S.Settings(t_min=0.0)
    img, t_final, load = gpu_forward(rast, upload(scene), cam, st)
    ref = oracle.render(scene, cam, st)
    keep = ref["near"] == 0
    assert ref["load"].max() == k and np.all(load[keep] == ref["load"][keep])
    assert np.count_nonzero(t_final[keep & (ref["load"] == k)] == 0.0) >= 8   # the underflow tested
    np.testing.assert_allclose(img[:, keep], ref["img"][:, keep], atol=1e-4)


def test_empty_scene_and_all_culled(rast):
    from paper_2409_08669_gb300.raster import upload
    cam = S.look_at((0, 0, -3), width=40, height=24)
    st = S.Settings(bg=(0.1, 0.2, 0.3))
    empty = S.tiny_scene(0, n=1).subset(np.arange(0))
    params = tuple(torch.zeros((0,) + a.shape[1:], dtype=torch.float32, device="cuda")
                   for a in empty.arrays())
    img, t_final, load = gpu_forward(rast, params, cam, st)
    assert rast.num_pairs() == 0
    np.testing.assert_array_equal(img, np.broadcast_to(np.float32([0.1, 0.2, 0.3])[:, None, None], img.shape))
    assert np.all(t_final == 1.0) and np.all(load == 0)
    behind = S.tiny_scene(1, n=500)
    behind.means[:, 2] = -5.0  # camera at z=-3 looking +z: all behind
    img, t_final, load = gpu_forward(rast, upload(behind), cam, st)
    assert rast.num_pairs() == 0 and np.all(load == 0)
    faint = S.tiny_scene(2, n=500)
    faint.opac[:] = np.float32(0.002)  # below 1/255: no pair in the adaptive modes
    gpu_forward(rast, upload(faint), cam, S.Settings(mode=S.MODE_AABB))
    assert rast.num_pairs() == 0
    gpu_forward(rast, upload(faint), cam, S.Settings(mode=S.MODE_PLAIN))
    assert rast.num_pairs() > 0


def test_capacity_overflow_is_reported_not_written():
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    r = Rasterizer(max_gaussians=20_000, pair_capacity=1000, max_width=256, max_height=256)
    try:
        scene = S.tiny_scene(0)
        cam = S.look_at((0, 0, -3), width=256, height=256)
        r.forward(upload(scene), cam, S.Settings())
        p, st = r.num_pairs(raise_on_error=False)
        assert st == _lib.ADR_ERR_CAPACITY
        assert p > 1000
        # the context stays usable
        small = S.tiny_scene(0, n=50)
        r.forward(upload(small), cam, S.Settings())
        assert r.num_pairs() <= 1000
    finally:
        r.close()


def test_invalid_arguments_rejected(rast):
    from paper_2409_08669_gb300 import _lib
    cam = S.look_at((0, 0, -3), width=4096, height=64)  # wider than the context allows
    scene = S.tiny_scene(0, n=10)
    from paper_2409_08669_gb300.raster import upload
    with pytest.raises(_lib.AdrError) as e:
        rast.forward(upload(scene), cam, S.Settings())
    assert e.value.status == _lib.ADR_ERR_INVALID
    cam = S.look_at((0, 0, -3), width=64, height=64)
    with pytest.raises(_lib.AdrError):
        rast.forward(upload(scene), cam, S.Settings(mode=7))
    with pytest.raises(_lib.AdrError) as e:
        rast.forward(upload(scene), cam, S.Settings(rect_rule=2))
    assert e.value.status == _lib.ADR_ERR_INVALID
    for near in (0.0, -1.0, float("inf")):   # the near plane must be in front of the camera
        with pytest.raises(_lib.AdrError) as e:
            rast.forward(upload(scene), S.look_at((0, 0, -3), width=64, height=64, near=near),
                         S.Settings())
        assert e.value.status == _lib.ADR_ERR_INVALID


def test_depth_slice_modes_render_identical_frames(rast):
    """The depth slices only skip Gaussians no pixel reaches: the image, T,
    l_i and the per-pixel list positions are bit-identical with and without."""
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    for scene, cam in ((S.tiny_scene(11, n=6000), S.look_at((0.3, -0.2, -2.2), width=250, height=190)),
                       (S.heavy_scene(n=200_000, seed=4), S.orbit_cameras(50, width=960, height=540)[9])):
        params = upload(scene)
        st = S.Settings(mode=S.MODE_AABB)
        out = []
        for mode in (Rasterizer.SLICES_NEVER, Rasterizer.SLICES_ALWAYS):
            rast.set_depth_slices(mode)
            img, t_final, load = rast.forward(params, cam, st)
            torch.cuda.synchronize()
            last, trav = rast.read_pixel_stats()
            out.append((img.cpu().numpy(), t_final.cpu().numpy(), load.cpu().numpy(), last, trav))
        rast.set_depth_slices(Rasterizer.SLICES_ADAPTIVE)
        for a, b in zip(*out):
            np.testing.assert_array_equal(a, b)
    from paper_2409_08669_gb300 import _lib
    with pytest.raises(_lib.AdrError):
        rast.set_depth_slices(7)


def test_heavy_cluster_frame_parity(rast):
    """A camera facing the heavy scene's dense cluster at 1080p: many tiles
    are still unfinished after depth slice 0 and their pixels blend ~900
    Gaussians each.  The sliced frame, with the last slice's tiles rendered
    whole or split into pixel halves across two CTAs (heavy tiles across
    CTAs), is bit-identical to the unsliced one (image, T, l_i, last and
    traversed positions), and the whole image keeps parity with the oracle
    in both."""
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    scene = S.heavy_scene(n=300_000, seed=2)
    cam = S.orbit_cameras(50, width=1920, height=1080)[0]
    st = S.Settings(mode=S.MODE_AABB)
    params = upload(scene)
    out = []
    for mode, split in ((Rasterizer.SLICES_NEVER, _lib.TILE_SPLIT_OFF),
                        (Rasterizer.SLICES_ALWAYS, _lib.TILE_SPLIT_OFF),
                        (Rasterizer.SLICES_ALWAYS, _lib.TILE_SPLIT_LAST_SLICE)):
        rast.set_depth_slices(mode)
        rast.set_tile_split(split)
        img, t_final, load = rast.forward(params, cam, st)
        torch.cuda.synchronize()
        last, trav = rast.read_pixel_stats()
        fc = rast.frame_counts()
        out.append((img.cpu().numpy(), t_final.cpu().numpy(), load.cpu().numpy(), last, trav))
        if mode == Rasterizer.SLICES_ALWAYS:
            assert fc["sliced"] == 1 and fc["visible_slice1"] > 0
    for other in out[1:]:
        for a, b in zip(out[0], other):
            np.testing.assert_array_equal(a, b)
    _check_frame(rast, scene, cam, st, "heavy300k-1080p/sliced/split")
    rast.set_tile_split(_lib.TILE_SPLIT_OFF)
    _check_frame(rast, scene, cam, st, "heavy300k-1080p/sliced")
    rast.set_depth_slices(Rasterizer.SLICES_ADAPTIVE)
    with pytest.raises(_lib.AdrError):
        rast.set_tile_split(3)


def test_degenerate_gaussians_are_culled(rast):
    """Gaussians with NaN centres or zero-norm rotations never reach a tile
    (their depth or det(Sigma') fails the cull), on both sides; the rest of the
    frame keeps parity with the oracle."""
    scene = S.tiny_scene(13, n=3000)
    scene.means[:6] = np.nan
    scene.rots[6:12] = 0.0
    cam = S.look_at((0, 0, -3), width=128, height=96)
    _check_frame(rast, scene, cam, S.Settings(mode=S.MODE_AABB), "degenerate")
    _, _, tiles = rast.read_gaussians()
    assert np.all(tiles[:12] == 0)
