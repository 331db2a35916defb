"""Failure detection without a GPU fault (bounded device waits).

Every device-side wait of the library is bounded: a decoupled-lookback wait
of the run-count scan that makes no progress for its poll limit gives up,
flags the frame and returns, and the frame's later stages skip their work.
adr_test_lookback_expiry makes one scan chunk withhold its prefix and lowers
the poll limit, so the next chunk's wait runs out on purpose (nothing hangs:
the wait gives up by construction).  Each test checks that the entry point
reports ADR_ERR_TIMEOUT, that the skipped frame holds only the background,
and that the next normal frame renders in parity with the oracle."""
import numpy as np
import pytest

import oracle
from paper_2409_08669_gb300 import scenes as S
from parity_utils import compare_images, gpu_forward

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture
def expiry():
    """Arms the hook for the test body; always restores normal operation."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300 import _lib
    yield lambda chunk=0, spins=64: _lib.adr_test_lookback_expiry(chunk, spins)
    _lib.adr_test_lookback_expiry(-1)


def _scene_and_camera():
    scene = S.tiny_scene(0)     # 10k Gaussians: >= 2 scan chunks of 4096 with tiles
    cam = S.look_at((0, 0, -3), width=256, height=256)
    return scene, cam, S.Settings(mode=S.MODE_AABB, bg=(0.25, 0.5, 0.75))


@pytest.mark.parametrize("slices", [0, 1], ids=["unsliced", "sliced"])
def test_context_frame_times_out_then_next_frame_is_in_parity(expiry, slices):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    scene, cam, st = _scene_and_camera()
    rast = Rasterizer(max_gaussians=1 << 15, pair_capacity=1 << 22, max_width=256, max_height=256)
    try:
        rast.set_depth_slices(slices)
        params = upload(scene)
        before, _, _ = gpu_forward(rast, params, cam, st)
        assert rast.sync_status() == _lib.ADR_OK
        _, _, tiles = rast.read_gaussians()
        assert int((tiles > 0).sum()) > 2 * 4096
        assert expiry(0, 64) == _lib.ADR_OK
        img, t_final, load = gpu_forward(rast, params, cam, st)
        assert rast.sync_status() == _lib.ADR_ERR_TIMEOUT
        assert "lookback" in _lib.last_error()
        bg = np.asarray(st.bg, np.float32)[:, None, None]
        assert np.array_equal(img, np.broadcast_to(bg, img.shape))   # the frame was skipped
        assert np.all(t_final == 1.0) and np.all(load == 0)
        assert expiry(-1) == _lib.ADR_OK
        img, t_final, load = gpu_forward(rast, params, cam, st)
        assert rast.sync_status() == _lib.ADR_OK
        assert np.array_equal(img, before)
        ref = oracle.render(scene, cam, st)
        compare_images(img, t_final, load, ref, ref["near"] != 0)
    finally:
        rast.close()


def test_server_request_times_out_and_the_server_recovers(expiry):
    from paper_2409_08669_gb300 import _lib
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    from paper_2409_08669_gb300.serve import Server
    scene, cam, st = _scene_and_camera()
    params = upload(scene)
    rast = Rasterizer(max_gaussians=1 << 15, pair_capacity=1 << 22, max_width=256, max_height=256)
    alone, _, _ = rast.forward(params, cam, st, want_aux=False)
    torch.cuda.synchronize()
    rast.close()
    srv = Server(max_slots=2, mem_budget_bytes=1 << 30, slot_pair_capacity=1 << 22,
                 slot_max_gaussians=1 << 15, max_width=256, max_height=256, use_graphs=False)
    try:
        sid = srv.add_scene(params, st)
        out = torch.full((3, 256, 256), -1.0, device="cuda")
        torch.cuda.synchronize()
        assert expiry(0, 64) == _lib.ADR_OK
        assert srv.poll(srv.submit(sid, cam, out)) == _lib.ADR_ERR_TIMEOUT
        assert "lookback" in _lib.last_error()
        assert expiry(-1) == _lib.ADR_OK
        out2 = torch.full((3, 256, 256), -1.0, device="cuda")
        torch.cuda.synchronize()
        assert srv.poll(srv.submit(sid, cam, out2)) == _lib.ADR_OK, _lib.last_error()
        assert torch.equal(out2, alone)
    finally:
        srv.close()
