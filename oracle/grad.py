"""Analytic gradients of the forward path — TEST INFRASTRUCTURE.

A plain FP64 PyTorch restatement of the per-Gaussian projection (Sec. 3.1,
Eq. 1-2 with the EWA covariance), the SH colour and the front-to-back blend
(Eq. 3) whose autograd gives the exact derivative of the implemented
function.  The discrete structure of a frame (which tiles each Gaussian
touches, the sorted per-tile lists, which pairs are skipped or stop a pixel)
is taken from the C oracle (`oracle/adr_oracle.c`) and the FP64 values
here, so the gradient follows the branches the forward path took.

The per-pixel load l_i (Eq. 12) is an integer count; its gradient uses the
straight-through reading d l_i / d alpha_ik = 1 for every blended pair,
so dL_load/d alpha_ik = dL/d l_i, or, with settings.load_grad = 1, for a
pixel that stopped early d l_i / d(-ln(1 - alpha_ik)) = -l_i / (-ln T_final)
(the paper does not say how L_load back-propagates; the tests pin the
straight-through reading to its definition and the early-stop reading to the
slope of the count l_i that the C oracle renders as opacities rise).

Only tests may import this module.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import F_VISIBLE, TILE, emit_pairs, preprocess, sort_pairs, tile_ranges


def _factorial(k):
    return float(math.factorial(k))


def real_sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real spherical harmonics Y_{l,m}(d), l <= degree, at unit directions
    d [..., 3], index l*l + l + m, Condon-Shortley phase.  Written in
    Cartesian form: Y = K Q_l^|m|(z) Re/Im((x + i y)^|m|) with Q_l^m the
    associated Legendre function divided by sin^m(theta), from the standard
    three-term recurrence, so it is a polynomial and differentiable everywhere."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    out = [None] * ((degree + 1) ** 2)
    # powers (x + i y)^m as (re, im)
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        r_prev, i_prev = re[-1], im[-1]
        re.append(r_prev * x - i_prev * y)
        im.append(r_prev * y + i_prev * x)
    for m in range(0, degree + 1):
        q_mm = (-1.0) ** m * float(np.prod(np.arange(1, 2 * m, 2))) if m > 0 else 1.0
        Q = {m: torch.full_like(z, q_mm)}
        if m + 1 <= degree:
            Q[m + 1] = z * (2 * m + 1) * q_mm
        for l in range(m + 2, degree + 1):
            Q[l] = ((2 * l - 1) * z * Q[l - 1] - (l + m - 1) * Q[l - 2]) / (l - m)
        for l in range(m, degree + 1):
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * _factorial(l - m) / _factorial(l + m))
            if m == 0:
                out[l * l + l] = K * Q[l]
            else:
                out[l * l + l + m] = math.sqrt(2.0) * K * Q[l] * re[m]
                out[l * l + l - m] = math.sqrt(2.0) * K * Q[l] * im[m]
    return torch.stack(out, dim=-1)


def _quat_rot(q):
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)
    return R


def gaussian_quantities(params, camera, settings):
    """Differentiable per-Gaussian pixel centre, conic, opacity and colour."""
    means, scales, rots, opac, sh = params
    rec = torch.as_tensor(camera.record(), dtype=torch.float64)
    V = rec[:16].reshape(4, 4)[:3, :3]
    t = rec[:16].reshape(4, 4)[:3, 3]
    fx, fy, cx, cy = rec[16], rec[17], rec[18], rec[19]
    cam_pos = rec[21:24]
    p = means @ V.T + t
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    R = _quat_rot(rots)
    M = R * scales[:, None, :]
    Sig = M @ M.transpose(1, 2)                       # Eq. 1
    limx = settings.jac_clamp * camera.width / (2.0 * float(fx))
    limy = settings.jac_clamp * camera.height / (2.0 * float(fy))
    txz = torch.clamp(x / z, -limx, limx) * z
    tyz = torch.clamp(y / z, -limy, limy) * z
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * txz / (z * z)], -1),
                     torch.stack([zero, fy / z, -fy * tyz / (z * z)], -1)], -2)
    T = J @ V
    C2 = T @ Sig @ T.transpose(1, 2)
    a = C2[:, 0, 0] + settings.lowpass
    b = C2[:, 0, 1]
    c = C2[:, 1, 1] + settings.lowpass
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    px = fx * x / z + cx
    py = fy * y / z + cy
    dvec = means - cam_pos
    dvec = dvec / torch.linalg.norm(dvec, dim=-1, keepdim=True)
    Y = real_sh_basis(dvec, settings.sh_degree)        # [N, nb]
    nb = (settings.sh_degree + 1) ** 2
    rgb = torch.clamp_min(torch.einsum("nk,nkc->nc", Y, sh[:, :nb, :]) + 0.5, 0.0)
    return px, py, conic, opac, rgb


def render_torch(params, camera, settings, structure=None):
    """img [3,H,W], T [H,W], straight-through load [H,W] in FP64 with autograd."""
    if structure is None:
        structure = frame_structure(params, camera, settings)
    px, py, conic, opac, rgb = gaussian_quantities(params, camera, settings)
    W, H = camera.width, camera.height
    tx = (W + TILE - 1) // TILE
    ranges, vals = structure["ranges"], structure["vals"]
    img = torch.zeros((3, H, W), dtype=torch.float64)
    Tout = torch.ones((H, W), dtype=torch.float64)
    load = torch.zeros((H, W), dtype=torch.float64)
    bg = torch.as_tensor(settings.bg, dtype=torch.float64)
    for tile in range(ranges.shape[0]):
        y0, x0 = (tile // tx) * TILE, (tile % tx) * TILE
        ys = torch.arange(y0, min(y0 + TILE, H), dtype=torch.float64)
        xs = torch.arange(x0, min(x0 + TILE, W), dtype=torch.float64)
        Yp, Xp = torch.meshgrid(ys, xs, indexing="ij")
        Yp, Xp = Yp.reshape(-1), Xp.reshape(-1)
        T = torch.ones_like(Xp)
        C = torch.zeros((3, Xp.shape[0]), dtype=torch.float64)
        L = torch.zeros_like(Xp)
        S = torch.zeros_like(Xp)    # optical depth of the blended Gaussians, sum of -ln(1 - alpha)
        done = torch.zeros(Xp.shape[0], dtype=torch.bool)
        for k in range(int(ranges[tile, 0]), int(ranges[tile, 1])):
            if bool(done.all()):
                break
            g = int(vals[k])
            dx, dy = px[g] - Xp, py[g] - Yp
            q = conic[g, 0] * dx * dx + 2 * conic[g, 1] * dx * dy + conic[g, 2] * dy * dy
            alpha = torch.clamp_max(opac[g] * torch.exp(-0.5 * q), 0.99)   # Eq. 2
            a_det = alpha.detach()
            live = (~done) & (a_det >= settings.alpha_low)
            test_T = T * (1 - alpha)
            stop = live & (test_T.detach() < settings.t_min)
            done = done | stop
            blend = live & ~stop
            bw = blend.to(torch.float64)
            C = C + rgb[g][:, None] * (alpha * T * bw)[None]                # Eq. 3
            T = torch.where(blend, test_T, T)
            L = L + bw * (1.0 + (alpha - a_det))                            # Eq. 12, straight-through
            S = S + bw * -torch.log1p(-alpha)
        if settings.load_grad == 1:
            # Pixels that stopped early: d l / d(-ln(1 - alpha_k)) = -l / (-ln T_final),
            # the count itself unchanged in value.
            cnt = L.detach()
            stopped = done & (cnt > 0)
            theta = S.detach().clamp_min(1e-300)
            L = torch.where(stopped, cnt - cnt / theta * (S - S.detach()), L)
        h, w = len(ys), len(xs)
        img[:, y0:y0 + h, x0:x0 + w] = (C + T[None] * bg[:, None]).reshape(3, h, w)
        Tout[y0:y0 + h, x0:x0 + w] = T.reshape(h, w)
        load[y0:y0 + h, x0:x0 + w] = L.reshape(h, w)
    return img, Tout, load


def clamp_near_pixels(scene, camera, settings, tol=1e-5):
    """[H,W] bool: pixels where a Gaussian that is blended (Eq. 3) has an
    unclamped opacity sigma * exp(-q/2) within `tol` (relative) of the 0.99
    clamp of Eq. 2.  The clamp switches that pair's opacity derivative off, so
    a path that evaluates the exponential with a relative error near `tol` may
    take the other side of min(0.99, .) there and differ by the whole term.
    Same traversal as render_torch, without autograd."""
    params = leaf_params(scene)
    structure = frame_structure(params, camera, settings)
    with torch.no_grad():
        px, py, conic, opac, _ = gaussian_quantities(params, camera, settings)
    W, H = camera.width, camera.height
    tx = (W + TILE - 1) // TILE
    ranges, vals = structure["ranges"], structure["vals"]
    out = np.zeros((H, W), bool)
    for tile in range(ranges.shape[0]):
        y0, x0 = (tile // tx) * TILE, (tile % tx) * TILE
        ys = torch.arange(y0, min(y0 + TILE, H), dtype=torch.float64)
        xs = torch.arange(x0, min(x0 + TILE, W), dtype=torch.float64)
        Yp, Xp = torch.meshgrid(ys, xs, indexing="ij")
        Yp, Xp = Yp.reshape(-1), Xp.reshape(-1)
        T = torch.ones_like(Xp)
        done = torch.zeros(Xp.shape[0], dtype=torch.bool)
        hit = torch.zeros(Xp.shape[0], dtype=torch.bool)
        for k in range(int(ranges[tile, 0]), int(ranges[tile, 1])):
            if bool(done.all()):
                break
            g = int(vals[k])
            dx, dy = px[g] - Xp, py[g] - Yp
            q = conic[g, 0] * dx * dx + 2.0 * conic[g, 1] * dx * dy + conic[g, 2] * dy * dy
            raw = opac[g] * torch.exp(-0.5 * q)
            alpha = torch.clamp_max(raw, 0.99)
            live = (~done) & (alpha >= settings.alpha_low)
            test_T = T * (1 - alpha)
            stop = live & (test_T < settings.t_min)
            done = done | stop
            blend = live & ~stop
            hit |= blend & (torch.abs(raw - 0.99) <= tol * 0.99)
            T = torch.where(blend, test_T, T)
        h, w = len(ys), len(xs)
        out[y0:y0 + h, x0:x0 + w] = hit.reshape(h, w).numpy()
    return out


class _ArrScene:
    def __init__(self, arrays):
        self.means, self.scales, self.rots, self.opac, self.sh = arrays

    @property
    def n(self):
        return self.means.shape[0]

    def arrays(self):
        return self.means, self.scales, self.rots, self.opac, self.sh


def frame_structure(params, camera, settings):
    """Tile lists from the C oracle at the same (detached) parameter values."""
    arrays = tuple(p.detach().cpu().numpy().astype(np.float64) for p in params)
    pre = preprocess(_ArrScene(arrays), camera, settings)
    keys, vals = emit_pairs(pre)
    skeys, svals = sort_pairs(keys, vals)
    ranges = tile_ranges(skeys, camera.width, camera.height)
    return dict(pre=pre, ranges=ranges, vals=svals)


def leaf_params(scene):
    return tuple(torch.tensor(np.asarray(a, np.float64), requires_grad=True) for a in scene.arrays())


def gradients(scene, camera, settings, dl_dimg, dl_dload=None):
    """dL/d(means, scales, rots, opac, sh) for L = <dl_dimg, img> + <dl_dload, load>."""
    params = leaf_params(scene)
    img, T, load = render_torch(params, camera, settings)
    L = (img * torch.as_tensor(dl_dimg, dtype=torch.float64)).sum()
    if dl_dload is not None:
        L = L + (load * torch.as_tensor(dl_dload, dtype=torch.float64)).sum()
    grads = torch.autograd.grad(L, params, allow_unused=True)
    out = []
    for p, g in zip(params, grads):
        out.append(np.zeros(p.shape) if g is None else g.numpy())
    return tuple(out), img.detach().numpy(), load.detach().numpy()


def visible_mask(pre):
    return (pre["flags"] & F_VISIBLE) != 0
