"""Image loss of the training objective — TEST INFRASTRUCTURE.

Plain FP64 numpy restatement of the L1 and SSIM terms of the total loss
(Sec. 4.4: lambda_L1 L1 + lambda_ssim L_ssim + lambda_load L_load) and of the
gradient of  w_l1 * mean|x - y| + w_ssim * (1 - mean SSIM)  with respect to
the rendered image x.

SSIM as defined by Wang, Bovik, Sheikh and Simoncelli (2004), the measure the
paper reports: per channel, local statistics under an 11x11 Gaussian window
of standard deviation 1.5 (normalised to sum 1),
    mu_x = w * x,  sigma_x^2 = w * x^2 - mu_x^2,  sigma_xy = w * (x y) - mu_x mu_y,
    S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1).  Reading: the window runs past the
border over zeros so the map has the image's size (the convention of 3DGS
training, on which the paper builds), and L_ssim = 1 - mean S.

The window sums are written out as the 121 shifted copies of the zero-padded
image, with no separable split; the gradient is the chain rule through the
three local moments mu_x, E[x^2], E[xy] and the adjoint of the window sum.
Only tests and __graft_entry__.smoke() may import this module (TEST
INFRASTRUCTURE: the product path never loads it).
"""
from __future__ import annotations

import numpy as np

RADIUS = 5
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The 11x11 Gaussian window (outer product of the 1-D taps), sum 1."""
    d = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-d * d / (2.0 * SIGMA * SIGMA))
    w2 = np.outer(g, g)
    return w2 / w2.sum()


def window_sum(a: np.ndarray) -> np.ndarray:
    """sum_{u,v} w[u, v] a[i + u - R, j + v - R] over a [H, W] plane padded with zeros."""
    w2 = window()
    h, wd = a.shape
    p = np.zeros((h + 2 * RADIUS, wd + 2 * RADIUS))
    p[RADIUS:RADIUS + h, RADIUS:RADIUS + wd] = a
    out = np.zeros((h, wd))
    for u in range(2 * RADIUS + 1):
        for v in range(2 * RADIUS + 1):
            out += w2[u, v] * p[u:u + h, v:v + wd]
    return out


def moments(x: np.ndarray, y: np.ndarray):
    """Local mu_x, mu_y, E[x^2], E[y^2], E[xy] of one channel."""
    return (window_sum(x), window_sum(y), window_sum(x * x), window_sum(y * y),
            window_sum(x * y))


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """S per element of [C, H, W] images (float64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.empty_like(x)
    for c in range(x.shape[0]):
        mx, my, exx, eyy, exy = moments(x[c], y[c])
        vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
        out[c] = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return out


def image_loss(x, y, w_l1=1.0, w_ssim=0.0, want_grad=True):
    """(mean |x - y|, mean SSIM, grad) with grad = d(w_l1 L1 + w_ssim (1 - SSIM)) / dx
    (L1 subgradient 0 where x == y); None if not want_grad."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    l1 = float(np.abs(x - y).mean())
    s_all = np.empty_like(x)
    grad = np.empty_like(x) if want_grad else None
    for c in range(x.shape[0]):
        mx, my, exx, eyy, exy = moments(x[c], y[c])
        vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
        a1, a2 = 2 * mx * my + C1, 2 * cxy + C2
        b1, b2 = mx * mx + my * my + C1, vx + vy + C2
        s = (a1 * a2) / (b1 * b2)
        s_all[c] = s
        if want_grad:
            # dS/d(mu_x, E[x^2], E[xy]) with sigma_x^2 = E[x^2] - mu_x^2, sigma_xy = E[xy] - mu_x mu_y
            d_mu = s * (2 * my / a1 - 2 * my / a2 - 2 * mx / b1 + 2 * mx / b2)
            d_xx = -s / b2
            d_xy = 2 * s / a2
            scale = -w_ssim / n                 # d (w_ssim (1 - mean S)) / dS at each element
            # adjoint of the zero-padded window sum (the window is symmetric)
            grad[c] = scale * (window_sum(d_mu) + 2 * x[c] * window_sum(d_xx)
                               + y[c] * window_sum(d_xy))
    if want_grad:
        grad += w_l1 / n * np.sign(x - y)
    return l1, float(s_all.mean()), grad
