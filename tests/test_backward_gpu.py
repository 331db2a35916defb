"""GPU backward (adr_render_backward, adr_load_loss) against the oracle's
analytic gradient (oracle/grad.py, pinned to finite differences of the FP64
oracle in tests/test_grad_oracle.py).

Bar: relative error of each gradient tensor, ||g_gpu - g_ref|| / ||g_ref||,
at most 1e-3, with the same seeded inputs.  (FP32 vs FP64: the recovered
transmittance T_k = T_{k+1} / (1 - alpha_k) and the atomic accumulation carry
~1e-6 relative error; a handful of near-threshold blend decisions can differ,
which the norm-wise bound absorbs.)"""
import numpy as np
import pytest

from oracle import grad as og
from paper_2409_08669_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("means", "scales", "rots", "opac", "sh")


@pytest.fixture(scope="module")
def rast():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300.raster import Rasterizer
    r = Rasterizer(max_gaussians=1 << 16, pair_capacity=1 << 22, max_width=256, max_height=256)
    yield r
    r.close()


def _scene(seed=5, n=2000, spread=0.6):
    sc = S.tiny_scene(seed, n=n)
    sc.means[:] = (sc.means * spread).astype(np.float32)
    return sc


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


def _gpu_grads(rast, sc, cam, st, w, v=None):
    from paper_2409_08669_gb300.raster import upload
    params = upload(sc)
    rast.forward(params, cam, st)
    dl_dimg = torch.tensor(w, dtype=torch.float32, device="cuda")
    dl_dload = None if v is None else torch.tensor(v, dtype=torch.float32, device="cuda")
    g = rast.backward(params, dl_dimg, dl_dload)
    torch.cuda.synchronize()
    assert rast.sync_status() == 0
    return [t.cpu().numpy().astype(np.float64) for t in g]


@pytest.mark.parametrize("mode", [S.MODE_AABB, S.MODE_PLAIN])
def test_backward_matches_oracle_gradient_2k_64px(rast, mode):
    """The 2k-Gaussian 64x64 sub-case of the training workload."""
    sc = _scene()
    cam = S.look_at((0.2, -0.1, -2.2), width=64, height=64)
    st = S.Settings(mode=mode)
    w = np.random.default_rng(1).normal(size=(3, 64, 64))
    got = _gpu_grads(rast, sc, cam, st, w)
    ref, _, _ = og.gradients(sc, cam, st, w)
    for name, a, b in zip(NAMES, got, ref):
        assert np.isfinite(a).all(), name
        assert _rel(a, b) <= 1e-3, (name, _rel(a, b))


@pytest.mark.parametrize("load_grad", [S.LOAD_GRAD_STRAIGHT, S.LOAD_GRAD_TERMINATION])
def test_backward_with_load_term_and_background(rast, load_grad):
    sc = _scene(seed=9, n=1500)
    cam = S.look_at((-0.3, 0.2, -2.4), width=80, height=48)
    st = S.Settings(mode=S.MODE_AABB, bg=(0.2, 0.5, 0.1), load_grad=load_grad)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(3, 48, 80))
    v = rng.normal(size=(48, 80)) * 0.05
    got = _gpu_grads(rast, sc, cam, st, w, v)
    ref, _, _ = og.gradients(sc, cam, st, w, dl_dload=v)
    for name, a, b in zip(NAMES, got, ref):
        assert _rel(a, b) <= 1e-3, (name, _rel(a, b))


def test_load_loss_kernel(rast):
    rng = np.random.default_rng(7)
    load = rng.integers(0, 60, size=(37, 53)).astype(np.int32)
    stats, grad = rast.load_loss(torch.tensor(load, device="cuda"), weight=0.45)
    torch.cuda.synchronize()
    mean, sd = load.mean(), load.std()
    assert stats[0].item() == pytest.approx(mean, rel=1e-12)
    assert stats[1].item() == pytest.approx(sd, rel=1e-12)
    np.testing.assert_allclose(grad.cpu().numpy(), 0.45 * (load - mean) / (load.size * sd), rtol=1e-5,
                               atol=1e-9)
    # constant load: zero gradient, zero std
    stats, grad = rast.load_loss(torch.full((8, 8), 3, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert stats[1].item() == 0.0 and torch.count_nonzero(grad).item() == 0


def test_autograd_function_matches_direct_backward(rast):
    from paper_2409_08669_gb300.autograd import load_balance_loss, rasterize
    from paper_2409_08669_gb300.raster import upload
    sc = _scene(seed=13, n=1200)
    cam = S.look_at((0.1, 0.1, -2.3), width=64, height=48)
    st = S.Settings(mode=S.MODE_AABB)
    params = [p.clone().requires_grad_(True) for p in upload(sc)]
    w = torch.randn((3, 48, 64), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    img, load_f, _ = rasterize(params, rast, cam, st)
    loss = (img * w).sum() + 0.45 * load_balance_loss(load_f, rast)
    loss.backward()
    stats, gl = rast.load_loss(load_f.detach().round().to(torch.int32), 0.45)
    direct = _gpu_grads(rast, sc, cam, st, w.cpu().numpy(), gl.cpu().numpy())
    for p, d, name in zip(params, direct, NAMES):
        np.testing.assert_allclose(p.grad.cpu().numpy(), d, rtol=1e-4, atol=1e-6, err_msg=name)


def test_training_steps_reduce_l1(rast):
    """A few Adam steps on raw parameters (log-scales, opacity logits) towards
    the render of a perturbed copy (means + N(0, 0.01), logits + N(0, 0.3))."""
    from paper_2409_08669_gb300.autograd import rasterize
    from paper_2409_08669_gb300.raster import upload
    base = _scene(seed=17, n=3000)
    target_scene = S.perturbed_scene(base, seed=4)
    cam = S.look_at((0.0, 0.1, -2.2), width=96, height=96)
    st = S.Settings(mode=S.MODE_AABB)
    tgt, _, _ = rast.forward(upload(target_scene), cam, st)
    tgt = tgt.clone()
    means, scales, rots, opac, sh = upload(base)
    raw = [means.clone().requires_grad_(True), torch.log(scales).requires_grad_(True),
           rots.clone().requires_grad_(True),
           torch.logit(opac.clamp(1e-4, 1 - 1e-4)).requires_grad_(True), sh.clone().requires_grad_(True)]
    opt = torch.optim.Adam(raw, lr=2e-3)
    losses = []
    for _ in range(25):
        opt.zero_grad()
        params = (raw[0], torch.exp(raw[1]), raw[2], torch.sigmoid(raw[3]), raw[4])
        img, _, _ = rasterize(params, rast, cam, st)
        loss = torch.abs(img - tgt).mean()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 0.8 * losses[0], losses
