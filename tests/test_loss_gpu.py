"""GPU parity of the image loss (adr_image_loss: L1 and SSIM terms of the total
loss, Sec. 4.4) against the FP64 oracle (oracle/ssim.py), through the C ABI.

Tolerance, from the arithmetic: the kernels form the local moments as
11 + 11-tap FP32 sums of values in [0, 1] (relative error ~1e-6) and the
variances as E[x^2] - mu^2, whose absolute error ~1e-7 is divided by
C2 = 9e-4, so S and its derivatives carry up to ~1e-4 relative error where the
local variance is small.  Means: |L1| within 1e-6 relative, mean SSIM within
2e-5 absolute.  Gradient: every element within 2e-3 of the largest oracle
element, and the error norm within 1e-3 of the gradient's norm.
"""
import numpy as np
import pytest

from oracle import ssim as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pair(seed, shape, noise=0.1, ties=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=shape).astype(np.float32)
    y = np.clip(x + rng.normal(0.0, noise, size=shape), 0.0, 1.0).astype(np.float32)
    if ties:
        idx = tuple(rng.integers(0, d, size=ties) for d in shape)
        y[idx] = x[idx]
    return x, y


def _gpu(x, y, w_l1, w_ssim):
    from paper_2409_08669_gb300.raster import image_loss
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    stats, grad = image_loss(xd, yd, w_l1, w_ssim)
    torch.cuda.synchronize()
    return stats.cpu().numpy(), grad.cpu().numpy().astype(np.float64)


def _check(x, y, w_l1, w_ssim):
    stats, g = _gpu(x, y, w_l1, w_ssim)
    l1, ms, go = O.image_loss(x, y, w_l1, w_ssim)
    assert stats[0] == pytest.approx(l1, rel=1e-6, abs=1e-12)
    assert abs(stats[1] - ms) <= 2e-5, (stats[1], ms)
    scale = np.abs(go).max()
    err = np.abs(g - go)
    assert err.max() <= 2e-3 * scale + 1e-12, (err.max(), scale)
    assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go) + 1e-12
    return stats, g, go


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("shape", [(3, 100, 130), (2, 33, 31), (1, 1, 1), (3, 5, 200), (1, 64, 64)])
@pytest.mark.parametrize("w", [(0.44, 0.11), (0.0, 1.0)])
def test_image_loss_parity_ragged(shape, w):
    x, y = _pair(sum(shape), shape, ties=3 if int(np.prod(shape)) > 10 else 0)
    _check(x, y, *w)


def test_image_loss_ties_and_identical_images():
    x, y = _pair(7, (3, 40, 50), ties=50)
    stats, g, go = _check(x, y, 1.0, 0.0)
    tied = x == y
    assert np.all(g[tied] == 0.0)
    stats, g = _gpu(x, x.copy(), 0.44, 0.11)
    assert stats[0] == 0.0 and abs(stats[1] - 1.0) <= 1e-5


def test_image_loss_parity_1080p_render_pair():
    """The training-size image (3 x 1080 x 1920): a render of the clustered
    scene against the render of its perturbed copy, as the fine-tune sees."""
    from paper_2409_08669_gb300 import scenes as S
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    base = S.cluster_scene(n=200_000, seed=1)
    target = S.perturbed_scene(base, seed=4)
    cam = S.orbit_cameras(50, width=1920, height=1080)[3]
    st = S.Settings(mode=S.MODE_AABB)
    rast = Rasterizer(max_gaussians=base.n, pair_capacity=1 << 26, max_width=1920, max_height=1080)
    try:
        a, _, _ = rast.forward(upload(base), cam, st, want_aux=False)
        a = a.clone()
        b, _, _ = rast.forward(upload(target), cam, st, want_aux=False)
        torch.cuda.synchronize()
        x, y = a.cpu().numpy(), b.cpu().numpy()
    finally:
        rast.close()
    stats, g, go = _check(x, y, 0.44, 0.11)
    print(f"1080p: L1={stats[0]:.6f} SSIM={stats[1]:.6f} max|dg|={np.abs(g - go).max():.2e} "
          f"max|g|={np.abs(go).max():.2e}")


def test_invalid_arguments_rejected():
    from paper_2409_08669_gb300 import _lib
    x = torch.zeros(3, 8, 8, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.AdrError) as e:
        _lib.adr_image_loss(x.data_ptr(), x.data_ptr(), 0, 8, 8, 1.0, 0.0, stats.data_ptr(), 0, 0, 0)
    assert e.value.status == _lib.ADR_ERR_INVALID
    with pytest.raises(_lib.AdrError):
        _lib.adr_image_loss(x.data_ptr(), x.data_ptr(), 3, 8, 8, 1.0, 0.0, stats.data_ptr(),
                            x.data_ptr(), 0, 0)   # gradient without scratch


def test_autograd_image_loss_backward():
    from paper_2409_08669_gb300.autograd import l1_ssim_loss
    x, y = _pair(9, (3, 48, 40))
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    loss = l1_ssim_loss(xd, torch.from_numpy(y).cuda(), 0.44, 0.11)
    (2.0 * loss).backward()
    l1, ms, go = O.image_loss(x, y, 0.44, 0.11)
    assert float(loss.detach()) == pytest.approx(0.44 * l1 + 0.11 * (1 - ms), rel=1e-5)
    g = xd.grad.cpu().numpy()
    assert np.abs(g - 2.0 * go).max() <= 4e-3 * np.abs(go).max()
