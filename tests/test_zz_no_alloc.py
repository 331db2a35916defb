"""The allocation-free frame entry point, called through the C ABI.

Callers that cannot allocate device memory while they render (for example a
host application whose GPU memory belongs to its own allocator, or a real-time
loop that cannot take an allocation's implicit synchronisation) use
adr_render_frame_noalloc, whose workspace is a static device array inside the
library.  This checks that it renders the same frame as the regular
context-based path (adr_preprocess + adr_sort + adr_render), on two calls in a
row, that it rejects sizes beyond its fixed limits, and that it reports a pair
overflow and an expired device wait with their own status, after which the
next call renders correctly again.  Collected last so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_08669_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(params, cam, st, img, t_final, load):
    from paper_2409_08669_gb300 import _lib
    lib = _lib.load()
    ptr = lambda t: ctypes.c_void_p(0 if t is None else t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.adr_render_frame_noalloc(*(ptr(p) for p in params), int(params[0].shape[0]),
                                          ctypes.byref(_lib.make_camera(cam)),
                                          ctypes.byref(_lib.make_settings(st)), ptr(img),
                                          ptr(t_final), ptr(load), stream)
    return status, lib.adr_last_error().decode()


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_noalloc_matches_context_path_twice(cuda):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload

    frames = [
        (S.tiny_scene(0), S.look_at((0, 0, -3), width=256, height=256), S.Settings(mode=S.MODE_AABB)),
        (S.tiny_scene(7, n=20_000), S.look_at((0.4, 0.2, -2.6), width=320, height=200),
         S.Settings(mode=S.MODE_PLAIN, bg=(0.2, 0.1, 0.0))),
    ]
    rast = Rasterizer(max_gaussians=32768, pair_capacity=1 << 20, max_width=512, max_height=512)
    try:
        for scene, cam, st in frames:
            params = upload(scene)
            ref_img, ref_t, ref_load = rast.forward(params, cam, st)
            img = torch.full((3, cam.height, cam.width), -1.0, device=cuda)
            t_final = torch.full((cam.height, cam.width), -1.0, device=cuda)
            load = torch.full((cam.height, cam.width), -1, dtype=torch.int32, device=cuda)
            status, msg = _noalloc(params, cam, st, img, t_final, load)
            assert status == _lib.ADR_OK, msg
            torch.cuda.synchronize()
            assert torch.max(torch.abs(img - ref_img)).item() <= 1e-4
            assert torch.max(torch.abs(t_final - ref_t)).item() <= 1e-4
            assert torch.equal(load, ref_load)
    finally:
        rast.close()


def test_noalloc_rejects_sizes_beyond_its_limits(cuda):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import upload
    scene = S.tiny_scene(0, n=40_000)   # more than 32768 Gaussians
    cam = S.look_at((0, 0, -3), width=64, height=64)
    img = torch.empty((3, 64, 64), device=cuda)
    status, msg = _noalloc(upload(scene), cam, S.Settings(), img, None, None)
    assert status == _lib.ADR_ERR_INVALID and "32768" in msg
    small = S.tiny_scene(0, n=100)
    big_cam = S.look_at((0, 0, -3), width=1024, height=64)   # wider than 512
    img = torch.empty((3, 64, 1024), device=cuda)
    status, msg = _noalloc(upload(small), big_cam, S.Settings(), img, None, None)
    assert status == _lib.ADR_ERR_INVALID


def _check_against_context_path(cuda, scene, cam, st):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    rast = Rasterizer(max_gaussians=32768, pair_capacity=1 << 20, max_width=512, max_height=512)
    try:
        params = upload(scene)
        ref_img, _, ref_load = rast.forward(params, cam, st)
        img = torch.full((3, cam.height, cam.width), -1.0, device=cuda)
        load = torch.full((cam.height, cam.width), -1, dtype=torch.int32, device=cuda)
        status, msg = _noalloc(params, cam, st, img, None, load)
        assert status == _lib.ADR_OK, msg
        torch.cuda.synchronize()
        assert torch.max(torch.abs(img - ref_img)).item() <= 1e-4
        assert torch.equal(load, ref_load)
    finally:
        rast.close()


def test_noalloc_reports_pair_overflow_as_capacity(cuda):
    """30k large Gaussians at 512x512 make several million Gaussian-tile pairs,
    more than the 2^20 the static scratch holds."""
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import upload
    scene = S.tiny_scene(3, n=30_000)
    scene.scales[:] = (scene.scales * 12.0).astype(np.float32)
    cam = S.look_at((0, 0, -3), width=512, height=512)
    img = torch.empty((3, 512, 512), device=cuda)
    status, msg = _noalloc(upload(scene), cam, S.Settings(mode=S.MODE_PLAIN), img, None, None)
    assert status == _lib.ADR_ERR_CAPACITY and "1048576" in msg, msg
    _check_against_context_path(cuda, S.tiny_scene(0), S.look_at((0, 0, -3), width=256, height=256),
                                S.Settings(mode=S.MODE_AABB))


def test_noalloc_reports_an_expired_device_wait_and_recovers(cuda):
    """The testing hook makes the run scan's lookback wait give up: the call
    returns ADR_ERR_TIMEOUT with the frame skipped (background only), and the
    next call renders as the context path does."""
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import upload
    scene = S.tiny_scene(0)
    cam = S.look_at((0, 0, -3), width=256, height=256)
    st = S.Settings(mode=S.MODE_AABB, bg=(0.5, 0.25, 0.125))
    img = torch.full((3, 256, 256), -1.0, device=cuda)
    try:
        assert _lib.adr_test_lookback_expiry(0, 64) == _lib.ADR_OK
        status, msg = _noalloc(upload(scene), cam, st, img, None, None)
    finally:
        _lib.adr_test_lookback_expiry(-1)
    assert status == _lib.ADR_ERR_TIMEOUT and "lookback" in msg, msg
    bg = torch.tensor(st.bg, device=cuda).view(3, 1, 1).expand(3, 256, 256)
    assert torch.equal(img, bg)
    _check_against_context_path(cuda, scene, cam, st)
