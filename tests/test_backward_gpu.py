"""GPU backward (adr_render_backward, adr_load_loss) against the oracle's
analytic gradient (oracle/grad.py, pinned to finite differences of the FP64
oracle in tests/test_grad_oracle.py).

Bar, element by element for every parameter of every Gaussian:
|g_gpu - g_ref| <= 1e-3 |g_ref| + 1e-3 max|g_ref| (the max over that
parameter tensor), with the same seeded inputs.  FP32 against FP64: the
recovered transmittance T_k = T_{k+1} / (1 - alpha_k) carries ~1e-5 relative
error after a hundred blends, and the warp sums and atomics add per-pixel
terms of both signs in FP32, whose rounding the absolute floor covers.
Pixels where a blend decision of the FP64 oracle lies within tolerance of
its threshold (alpha vs alpha_low, T(1 - alpha) vs t_min, and a blended
pair's opacity at the 0.99 clamp) get a zero upstream gradient, so the side
FP32 takes there cannot change any gradient; these are the forward tests'
near-threshold pixels.

Cases: uniform scenes at 64x64 and 80x48, and a dense cluster at 136x120
(lists of up to ~3.5k Gaussians per tile, ~50 blended per pixel), where many
pixels of a warp blend the same Gaussian and the warp-reduce-then-atomic
accumulation runs under contention."""
import numpy as np
import pytest

import oracle
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


def _dense_scene(seed=21, n=6000):
    """All Gaussians in the heavy scene's dense cluster (means N(0, 0.22),
    log-scales N(-3, 0.7)), seen from distance ~1.5 so it fills the image."""
    return S.heavy_scene(n=n, seed=seed, dense_fraction=1.0)


def _near_pixels(sc, cam, st):
    ref = oracle.render(sc, cam, st)
    return (ref["near"] != 0) | og.clamp_near_pixels(sc, cam, st)


def _check_elementwise(got, ref, label):
    for name, a, b in zip(NAMES, got, ref):
        assert np.isfinite(a).all(), (label, name)
        a, b = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
        err = np.abs(a - b)
        tol = 1e-3 * np.abs(b) + 1e-3 * np.abs(b).max()
        bad = err > tol
        if bad.any():
            i, j = np.argwhere(bad)[0]
            raise AssertionError(f"{label}/{name}: {int(bad.sum())} of {b.size} elements differ; "
                                 f"first Gaussian {i} [{j}]: gpu {a[i, j]:.6e} oracle {b[i, j]:.6e} "
                                 f"(max|oracle| {np.abs(b).max():.3e})")


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
    w[:, _near_pixels(sc, cam, st)] = 0.0
    got = _gpu_grads(rast, sc, cam, st, w)
    ref, _, _ = og.gradients(sc, cam, st, w)
    _check_elementwise(got, ref, f"2k-64px/{S.MODE_NAMES[mode]}")


@pytest.mark.parametrize("load_grad", [S.LOAD_GRAD_STRAIGHT, S.LOAD_GRAD_TERMINATION])
def test_backward_with_load_term_and_background(rast, load_grad):
    sc = _scene(seed=9, n=1500)
    cam = S.look_at((-0.3, 0.2, -2.4), width=80, height=48)
    st = S.Settings(mode=S.MODE_AABB, bg=(0.2, 0.5, 0.1), load_grad=load_grad)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(3, 48, 80))
    v = rng.normal(size=(48, 80)) * 0.05
    near = _near_pixels(sc, cam, st)
    w[:, near] = 0.0
    v[near] = 0.0
    got = _gpu_grads(rast, sc, cam, st, w, v)
    ref, _, _ = og.gradients(sc, cam, st, w, dl_dload=v)
    _check_elementwise(got, ref, f"load-term/{load_grad}")


@pytest.mark.parametrize("mode,load_grad", [(S.MODE_AABB, None), (S.MODE_PLAIN, None),
                                            (S.MODE_AABB, S.LOAD_GRAD_TERMINATION)])
def test_backward_dense_cluster_elementwise(rast, mode, load_grad):
    """6000 Gaussians of the dense cluster at 136x120 (ragged last tile row and
    column): hundreds to thousands of Gaussians per tile list, up to ~130
    blended per pixel, so every warp reduces and atomically adds the
    gradients of Gaussians that most of its pixels blend."""
    sc = _dense_scene()
    cam = S.look_at((0.3, -0.2, -1.5), width=136, height=120)
    st = S.Settings(mode=mode, bg=(0.05, 0.1, 0.2),
                    load_grad=S.LOAD_GRAD_STRAIGHT if load_grad is None else load_grad)
    rng = np.random.default_rng(8)
    w = rng.normal(size=(3, 120, 136))
    v = None if load_grad is None else rng.normal(size=(120, 136)) * 0.02
    near = _near_pixels(sc, cam, st)
    w[:, near] = 0.0
    if v is not None:
        v[near] = 0.0
    got = _gpu_grads(rast, sc, cam, st, w, v)
    ref, _, load = og.gradients(sc, cam, st, w, dl_dload=v)
    assert load.max() >= 80, "the case must blend many Gaussians per pixel"
    _check_elementwise(got, ref, f"dense/{S.MODE_NAMES[mode]}/{load_grad}")


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
