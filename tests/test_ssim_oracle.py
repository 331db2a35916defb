"""Pins of the oracle's image loss (L1 + SSIM, the image terms of the total loss
in Sec. 4.4) against things other than itself: scipy's Gaussian filter for the
window sums, closed forms for identical and constant images, the symmetry and
bound of SSIM, a per-pixel double loop, and central finite differences of the
loss for the gradient."""
import math

import numpy as np
import pytest

from oracle import ssim as O


def _pair(seed, shape=(2, 19, 23), noise=0.1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=shape)
    y = np.clip(x + rng.normal(0.0, noise, size=shape), 0.0, 1.0)
    return x, y


def test_window_sum_matches_scipy_gaussian_filter():
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(0)
    a = rng.normal(size=(17, 26))
    # radius = int(truncate * sigma + 0.5) = 5 taps each side, zeros past the border
    ref = gaussian_filter(a, sigma=1.5, truncate=10.0 / 3.0, mode="constant", cval=0.0)
    np.testing.assert_allclose(O.window_sum(a), ref, rtol=0, atol=1e-13)
    assert O.window().sum() == pytest.approx(1.0, abs=1e-15)


def test_window_sum_per_pixel_double_loop():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(9, 12))
    got = O.window_sum(a)
    for (i, j) in [(0, 0), (4, 7), (8, 11), (2, 10)]:
        acc = 0.0
        for u in range(-5, 6):
            for v in range(-5, 6):
                if 0 <= i + u < 9 and 0 <= j + v < 12:
                    acc += math.exp(-(u * u + v * v) / (2 * 1.5 ** 2)) * a[i + u, j + v]
        norm = sum(math.exp(-(u * u) / 4.5) for u in range(-5, 6)) ** 2
        assert got[i, j] == pytest.approx(acc / norm, abs=1e-14)


def test_identical_images_give_ssim_one_and_zero_l1():
    x, _ = _pair(2)
    s = O.ssim_map(x, x)
    np.testing.assert_allclose(s, 1.0, rtol=0, atol=1e-12)
    l1, ms, _ = O.image_loss(x, x, 1.0, 1.0)
    assert l1 == 0.0 and ms == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("a,b", [(0.2, 0.7), (0.9, 0.1), (0.5, 0.5)])
def test_constant_images_interior_closed_form(a, b):
    """Away from the border the window sees only the constants: no variance,
    so S = (2ab + C1) / (a^2 + b^2 + C1)."""
    x = np.full((1, 16, 18), a)
    y = np.full((1, 16, 18), b)
    s = O.ssim_map(x, y)[0]
    want = (2 * a * b + 0.01 ** 2) / (a * a + b * b + 0.01 ** 2)
    np.testing.assert_allclose(s[5:-5, 5:-5], want, rtol=1e-11)   # E[x^2] - mu^2 rounds to ~1e-17, over C2


@pytest.mark.parametrize("a,d,b", [(0.5, 0.3, 0.2), (0.4, 0.05, 0.9)])
def test_checkerboard_against_constant_closed_form(a, d, b):
    """x = a + d (-1)^(i+j) against the constant b.  Away from the border the
    window's mean of x is a + d s (-1)^(i+j), with s = (sum_u g_u (-1)^u /
    sum_u g_u)^2 for the 1-D taps g_u = exp(-u^2 / (2 * 1.5^2)), |u| <= 5; its
    variance is d^2 (1 - s^2); the covariance with a constant is 0.  So
    S = (2 mu_x b + C1) C2 / ((mu_x^2 + b^2 + C1) (d^2 (1 - s^2) + C2)),
    which, unlike the constant-image case, depends on C2."""
    h, w = 16, 18
    ii, jj = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    sign = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    x = (a + d * sign)[None]
    y = np.full((1, h, w), b)
    g = [math.exp(-u * u / (2 * 1.5 ** 2)) for u in range(-5, 6)]
    s = (sum(gu * (-1) ** u for gu, u in zip(g, range(-5, 6))) / sum(g)) ** 2
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    mu = a + d * s * sign
    want = (2 * mu * b + c1) * c2 / ((mu * mu + b * b + c1) * (d * d * (1 - s * s) + c2))
    got = O.ssim_map(x, y)[0]
    np.testing.assert_allclose(got[5:-5, 5:-5], want[5:-5, 5:-5], rtol=1e-9)


def test_ssim_symmetric_and_bounded():
    x, y = _pair(3)
    s_xy, s_yx = O.ssim_map(x, y), O.ssim_map(y, x)
    np.testing.assert_allclose(s_xy, s_yx, rtol=0, atol=1e-14)
    assert np.all(s_xy <= 1.0 + 1e-12) and np.all(s_xy > -1.0)
    assert O.image_loss(x, y, 0.0, 1.0)[1] < 1.0 - 1e-3
    # anti-correlated structure: negative local covariance lowers S below the
    # value the means alone give
    z = 1.0 - x
    assert O.ssim_map(x, z).mean() < O.ssim_map(x, x + 0.0 * z).mean()


@pytest.mark.parametrize("w_l1,w_ssim", [(0.0, 1.0), (1.0, 0.0), (0.44, 0.11)])
def test_gradient_matches_central_differences(w_l1, w_ssim):
    x, y = _pair(4, shape=(2, 9, 11))
    _, _, g = O.image_loss(x, y, w_l1, w_ssim)

    def loss(xx):
        l1, s, _ = O.image_loss(xx, y, w_l1, w_ssim, want_grad=False)
        return w_l1 * l1 + w_ssim * (1.0 - s)

    rng = np.random.default_rng(5)
    h = 1e-6
    for idx in [tuple(rng.integers(0, d) for d in x.shape) for _ in range(25)] + [(0, 0, 0), (1, 8, 10)]:
        if abs(x[idx] - y[idx]) < 10 * h:
            continue   # the L1 kink
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(xp) - loss(xm)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10), idx


def test_l1_subgradient_zero_at_ties():
    x, y = _pair(6, shape=(1, 8, 8))
    y[0, 3, 3] = x[0, 3, 3]
    _, _, g = O.image_loss(x, y, 1.0, 0.0)
    assert g[0, 3, 3] == 0.0
    assert abs(g[0, 2, 2]) == pytest.approx(1.0 / x.size)
