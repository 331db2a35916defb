"""adr_render_host: the frame from HOST buffers.  Pinned buffers mapped into
the device's address space are read (and the outputs written) in place;
other host memory, or ADR_HOST_READ_COPY, goes through device staging
copies.  Both give the same frame as the device-pointer path."""
import numpy as np
import pytest

from paper_2409_08669_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rast():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300.raster import Rasterizer
    r = Rasterizer(max_gaussians=1 << 18, pair_capacity=1 << 24, max_width=1280, max_height=720)
    yield r
    r.close()


def _host_frame(rast, scene, cam, st, pinned):
    from paper_2409_08669_gb300 import _lib
    wrap = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()) if pinned else \
        (lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()))
    arrays = [wrap(a) for a in scene.arrays()]
    img = wrap(np.zeros((3, cam.height, cam.width), np.float32))
    t_final = wrap(np.zeros((cam.height, cam.width), np.float32))
    load = wrap(np.zeros((cam.height, cam.width), np.int32))
    stream = torch.cuda.current_stream().cuda_stream
    _lib.adr_render_host(rast.ctx, *[a.data_ptr() for a in arrays], scene.n, _lib.make_camera(cam),
                         _lib.make_settings(st), img.data_ptr(), t_final.data_ptr(), load.data_ptr(),
                         stream)
    return img.numpy().copy(), t_final.numpy().copy(), load.numpy().copy()


def test_host_frames_match_device_frame(rast):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import upload
    scene = S.cluster_scene(n=150_000, seed=3)
    cam = S.orbit_cameras(50, width=1280, height=720)[11]
    st = S.Settings(mode=S.MODE_AABB)
    from paper_2409_08669_gb300.raster import Rasterizer
    img, t_final, load = rast.forward(upload(scene), cam, st)
    torch.cuda.synchronize()
    ref = (img.cpu().numpy(), t_final.cpu().numpy(), load.cpu().numpy())
    frames = {}
    # with depth slices the mapped path defers the SH colours to each Render
    # launch; without, Preprocess reads them
    for slices in (Rasterizer.SLICES_ALWAYS, Rasterizer.SLICES_NEVER):
        rast.set_depth_slices(slices)
        for mode in (_lib.HOST_READ_MAPPED, _lib.HOST_READ_COPY):
            _lib.adr_set_host_reads(rast.ctx, mode)
            for pinned in (True, False):
                frames[(slices, mode, pinned)] = _host_frame(rast, scene, cam, st, pinned)
    rast.set_depth_slices(Rasterizer.SLICES_ADAPTIVE)
    _lib.adr_set_host_reads(rast.ctx, _lib.HOST_READ_MAPPED)
    for key, out in frames.items():
        for a, b in zip(out, ref):
            np.testing.assert_array_equal(a, b, err_msg=str(key))
    with pytest.raises(_lib.AdrError):
        _lib.adr_set_host_reads(rast.ctx, 5)
