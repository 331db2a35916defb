"""Serving scheduler (adr_serve_*): continuous batching over resident scenes.

Each request's image must be bit-identical to the same frame rendered alone
through adr_preprocess + adr_sort + adr_render (the kernels are the same and
deterministic), whether it ran alone or overlapped with other requests, with
graph replay or plain launches; and served images must match the CPU oracle
within the forward tests' bar (1e-4 per channel off near-threshold pixels)."""
import numpy as np
import pytest

import oracle
from paper_2409_08669_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    scenes = [S.cluster_scene(60_000, seed=3), S.tiny_scene(8, n=6000), S.heavy_scene(120_000, seed=5)]
    params = [upload(sc) for sc in scenes]
    settings = [S.Settings(mode=S.MODE_AABB), S.Settings(mode=S.MODE_PLAIN, bg=(0.1, 0.2, 0.3)),
                S.Settings(mode=S.MODE_CIRCLE)]
    rng = np.random.default_rng(11)
    sizes = [(320, 240), (256, 256), (200, 136), (480, 270)]
    reqs = []
    for k in range(24):
        sid = int(rng.integers(0, len(scenes)))
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        radius = 4.0 if sid != 1 else 2.5
        reqs.append((sid, S.sphere_camera(rng, radius=radius, width=w, height=h)))
    rast = Rasterizer(max_gaussians=1 << 18, pair_capacity=1 << 23, max_width=512, max_height=512)
    alone = []
    for sid, cam in reqs:
        img, _, _ = rast.forward(params[sid], cam, settings[sid], want_aux=False)
        alone.append(img.clone())
    torch.cuda.synchronize()
    assert rast.sync_status() == 0
    rast.close()
    yield dict(scenes=scenes, params=params, settings=settings, reqs=reqs, alone=alone)


def _server(**kw):
    from paper_2409_08669_gb300.serve import Server
    cfg = dict(max_slots=4, mem_budget_bytes=4 << 30, slot_pair_capacity=1 << 23,
               slot_max_gaussians=1 << 18, max_width=512, max_height=512)
    cfg.update(kw)
    return Server(**cfg)


def _register(srv, env):
    return [srv.add_scene(p, st) for p, st in zip(env["params"], env["settings"])]


@pytest.mark.parametrize("use_graphs,max_batch", [(True, 1), (False, 1), (True, 4), (False, 4)])
def test_mix_equals_alone_bit_exact(env, use_graphs, max_batch):
    """Batched (max_batch 4: two groups of four slots, each batch one
    Preprocess and one Render launch per depth slice over its cameras) or not,
    every served image equals its frame rendered alone."""
    from paper_2409_08669_gb300 import _lib
    srv = _server(use_graphs=use_graphs, max_batch=max_batch, max_slots=8 if max_batch > 1 else 4)
    ids = _register(srv, env)
    torch.cuda.synchronize()
    outs, tickets = [], []
    for sid, cam in env["reqs"]:          # all submitted at once: they overlap
        out = torch.full((3, cam.height, cam.width), -1.0, device="cuda")
        outs.append(out)
    torch.cuda.synchronize()
    for (sid, cam), out in zip(env["reqs"], outs):
        tickets.append(srv.submit(ids[sid], cam, out))
    for t in tickets:
        assert srv.poll(t) == _lib.ADR_OK, _lib.last_error()
    for k, (out, ref) in enumerate(zip(outs, env["alone"])):
        assert torch.equal(out, ref), f"request {k} differs from its frame rendered alone"
    st = srv.stats()
    assert st["completed"] == len(tickets)
    assert st["max_inflight"] > 1 and st["admitted_while_busy"] > 0, st
    if use_graphs:
        assert st["graph_replays"] == st["batches"]
    if max_batch > 1:
        assert st["largest_batch"] > 1 and st["mean_batch"] > 1.0, st
        assert st["batches"] < len(tickets)
    else:
        assert st["largest_batch"] == 1 and st["batches"] == len(tickets)
    # second pass: graphs replayed from the cache for other cameras give the same images
    outs2 = [torch.empty_like(o) for o in outs]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[sid], cam, o) for (sid, cam), o in zip(env["reqs"], outs2)]
    for t in tickets:
        assert srv.poll(t) == _lib.ADR_OK, _lib.last_error()
    for out, ref in zip(outs2, env["alone"]):
        assert torch.equal(out, ref)
    srv.close()


@pytest.mark.parametrize("slots,budget", [(1, 4 << 30), (4, 30 << 20)])
def test_single_slot_or_tight_budget_serialise(env, slots, budget):
    """One frame in flight at a time -- one slot, or a budget below two
    predicted frames of the 120k-Gaussian scene (150 B x 120k = 18 MB each):
    the same images, never more than one frame in flight."""
    from paper_2409_08669_gb300 import _lib
    srv = _server(max_slots=slots, mem_budget_bytes=budget, slot_pair_capacity=1 << 21)
    ids = _register(srv, env)
    torch.cuda.synchronize()
    sel = [k for k, (s, _) in enumerate(env["reqs"]) if s == 2][:6]
    assert len(sel) >= 3
    outs = [torch.empty((3, env["reqs"][k][1].height, env["reqs"][k][1].width), device="cuda")
            for k in sel]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[2], env["reqs"][k][1], o) for k, o in zip(sel, outs)]
    for t in tickets:
        assert srv.poll(t) == _lib.ADR_OK, _lib.last_error()
    for k, out in zip(sel, outs):
        assert torch.equal(out, env["alone"][k])
    assert srv.stats()["max_inflight"] == 1
    srv.close()


def test_admission_rejects_request_that_never_fits(env):
    from paper_2409_08669_gb300 import _lib
    srv = _server(mem_budget_bytes=1 << 20)      # 1 MiB < 150 B x 60k Gaussians
    ids = _register(srv, env)
    sid, cam = env["reqs"][0]
    out = torch.empty((3, cam.height, cam.width), device="cuda")
    assert srv.submit_status(ids[0], cam, out) == _lib.ADR_ERR_ADMISSION
    assert srv.stats()["rejected"] == 1
    assert srv.submit_status(99, cam, out) == _lib.ADR_ERR_INVALID
    srv.close()


def test_poll_pending_timeout_and_unknown_ticket(env):
    from paper_2409_08669_gb300 import _lib
    srv = _server(max_slots=1)
    ids = _register(srv, env)
    cams = [S.sphere_camera(np.random.default_rng(k), width=480, height=270) for k in range(12)]
    outs = [torch.empty((3, 270, 480), device="cuda") for _ in cams]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[2], c, o) for c, o in zip(cams, outs)]
    last = tickets[-1]
    assert srv.poll(last, 0) == _lib.ADR_PENDING
    assert srv._lib.adr_serve_poll(srv._h, last, -5) == _lib.ADR_ERR_INVALID
    assert srv.poll(last, 1) in (_lib.ADR_ERR_TIMEOUT, _lib.ADR_OK)
    for t in tickets:
        st = srv.poll(t)
        assert st == _lib.ADR_OK or (t == last and st == _lib.ADR_ERR_INVALID)
    assert srv.poll(12345678, 0) == _lib.ADR_ERR_INVALID
    srv.close()


def test_capacity_overflow_reported_and_server_recovers(env):
    from paper_2409_08669_gb300 import _lib
    srv = _server(slot_pair_capacity=1 << 12)
    ids = _register(srv, env)
    sid, cam = next((s, c) for s, c in env["reqs"] if s == 0)
    out = torch.empty((3, cam.height, cam.width), device="cuda")
    torch.cuda.synchronize()
    t = srv.submit(ids[0], cam, out)
    assert srv.poll(t) == _lib.ADR_ERR_CAPACITY
    assert srv.stats()["capacity_errors"] == 1
    # a frame that fits still renders correctly afterwards
    small = S.look_at((0.0, 0.0, -2.5), width=32, height=32)
    tiny = S.tiny_scene(1, n=50)
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    p = upload(tiny)
    sid2 = srv.add_scene(p, S.Settings())
    r = Rasterizer(max_gaussians=1024, pair_capacity=1 << 12, max_width=64, max_height=64)
    ref, _, _ = r.forward(p, small, S.Settings(), want_aux=False)
    torch.cuda.synchronize()
    out2 = torch.empty((3, 32, 32), device="cuda")
    t = srv.submit(sid2, small, out2)
    assert srv.poll(t) == _lib.ADR_OK
    assert torch.equal(out2, ref)
    r.close()
    srv.close()


def _near_tiles_mask(pre, width, height, pad=1):
    """Pixels of the tiles (grown by `pad` tiles) of Gaussians whose cull or
    tile decision the oracle flags as within tolerance of its threshold: the
    CUDA path may give such a Gaussian a different tile set."""
    tx, ty = (width + 15) // 16, (height + 15) // 16
    m = np.zeros((height, width), bool)
    near = ((pre["flags"] & oracle.F_NEAR) != 0) & (pre["tiles"] > 0)
    for g in np.nonzero(near)[0]:
        x0, y0, x1, y1 = pre["rect"][g]
        x0, y0 = max(0, x0 - pad), max(0, y0 - pad)
        x1, y1 = min(tx, x1 + pad), min(ty, y1 + pad)
        m[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    return m


@pytest.mark.parametrize("use_graphs,max_batch", [(True, 1), (False, 1), (True, 4)])
def test_served_images_match_the_oracle(env, use_graphs, max_batch):
    """One request of each resident scene (AABB, PLAIN with a background,
    CIRCLE), served while the other requests overlap with it (batched with
    them when max_batch > 1), against the FP64 oracle on the same scene,
    camera and settings."""
    from paper_2409_08669_gb300 import _lib
    srv = _server(use_graphs=use_graphs, max_batch=max_batch, max_slots=8 if max_batch > 1 else 4)
    ids = _register(srv, env)
    pick = {}
    for k, (sid, _) in enumerate(env["reqs"]):
        pick.setdefault(sid, k)
    assert sorted(pick) == [0, 1, 2]
    outs = [torch.full((3, cam.height, cam.width), -1.0, device="cuda") for _, cam in env["reqs"]]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[sid], cam, o) for (sid, cam), o in zip(env["reqs"], outs)]
    for t in tickets:
        assert srv.poll(t) == _lib.ADR_OK, _lib.last_error()
    assert srv.stats()["max_inflight"] > 1
    srv.close()
    for sid, k in sorted(pick.items()):
        cam = env["reqs"][k][1]
        img = outs[k].cpu().numpy().astype(np.float64)
        ref = oracle.render(env["scenes"][sid], cam, env["settings"][sid])
        exclude = (ref["near"] != 0) | _near_tiles_mask(ref["pre"], cam.width, cam.height)
        err = np.abs(img - ref["img"]).max(axis=0)
        bad = (err > 1e-4) & ~exclude
        assert not bad.any(), (f"scene {sid} request {k}: {int(bad.sum())} pixels differ from the "
                               f"oracle by up to {err[bad].max():.2e}")
        assert int((err > 1e-4).sum()) <= max(4, 1e-4 * cam.width * cam.height)
        assert float(err[~exclude].max()) <= 1e-4
