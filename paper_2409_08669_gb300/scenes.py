"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras and render settings.

This module only draws random numbers and lays them out; it holds none of the
rasterization arithmetic (no projection, covariance, culling or blending).  Both
the CUDA path and the CPU oracle receive exactly the arrays built here.

Layout (all float32, C-contiguous, structure of arrays):
    means  [N, 3]      world-space centres X0 (Sec. 3.1, Eq. 1)
    scales [N, 3]      activated per-axis scales s (positive)
    rots   [N, 4]      rotation quaternion (w, x, y, z), not necessarily unit
    opac   [N]         activated opacity sigma in (0, 1)
    sh     [N, 16, 3]  SH coefficients, index l*l + l + m, colour channel last

Camera record (float32[24]): view[16] (row-major world->camera, OpenCV axes:
x right, y down, z forward), fx, fy, cx, cy, near, cam_pos[3].  Pixel (i, j)
has its centre at integer coordinates; cx = (W-1)/2, cy = (H-1)/2.

Workload recipes follow the paper's setting (Sec. 5.1: real captured scenes of
~1-3M Gaussians on one GPU) with synthetic stand-ins for its datasets:
  * tiny: 10k Gaussians uniform in [-1,1]^3, 256x256, one camera at distance 3;
  * clustered: 90% in 64 anisotropic clusters + 10% uniform background;
  * heavy: 30% of the Gaussians in one dense central cluster.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MODE_PLAIN = 0
MODE_CIRCLE = 1
MODE_AABB = 2
MODE_NAMES = {MODE_PLAIN: "plain", MODE_CIRCLE: "adr_circle", MODE_AABB: "adr_aabb"}

# Tile-rectangle rules: the pixel-conservative rule (lossless, the default) and
# the original 3DGS rasterizer's rounding (for comparison with 3DGS renders).
RECT_PIXEL = 0
RECT_3DGS = 1

# Readings of d l_i / d alpha for the load-balancing loss: straight-through
# (the default) or through the early stop of pixels that terminated.
LOAD_GRAD_STRAIGHT = 0
LOAD_GRAD_TERMINATION = 1

CAMERA_FLOATS = 24


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    rots: np.ndarray
    opac: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.means, self.scales, self.rots, self.opac, self.sh)))

    def arrays(self):
        return self.means, self.scales, self.rots, self.opac, self.sh

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays())


@dataclasses.dataclass
class Camera:
    """Pinhole camera; `record()` gives the float32[24] layout described above."""
    view: np.ndarray  # float32[4, 4]
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    cam_pos: np.ndarray  # float32[3]
    width: int
    height: int

    def record(self) -> np.ndarray:
        r = np.zeros(CAMERA_FLOATS, np.float32)
        r[:16] = self.view.reshape(-1)
        r[16:21] = (self.fx, self.fy, self.cx, self.cy, self.near)
        r[21:24] = self.cam_pos
        return r


@dataclasses.dataclass
class Settings:
    """Render settings; every value is float32-representable so both sides
    threshold against the identical number."""
    mode: int = MODE_AABB
    alpha_low: float = float(np.float32(1.0 / 255.0))  # minimum splatting opacity (Sec. 5.1.2)
    t_min: float = float(np.float32(1e-4))             # early-termination transmittance
    lowpass: float = float(np.float32(0.3))            # screen-space dilation of Sigma'
    jac_clamp: float = float(np.float32(1.3))          # Jacobian clamp, in units of tan(fov/2)
    bg: tuple = (0.0, 0.0, 0.0)
    sh_degree: int = 3
    rect_rule: int = RECT_PIXEL
    load_grad: int = LOAD_GRAD_STRAIGHT

    def with_mode(self, mode: int) -> "Settings":
        return dataclasses.replace(self, mode=mode)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), width=256, height=256,
            fovx_deg=60.0, near=0.2) -> Camera:
    """World->camera view with rows (right, down, forward); fx = fy from FOVx."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    u = np.asarray(up, np.float64)
    r = np.cross(f, u)
    if np.linalg.norm(r) < 1e-6:  # looking along the up axis: pick another up
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f])
    view = np.eye(4)
    view[:3, :3] = rot
    view[:3, 3] = -rot @ eye
    fx = width / (2.0 * math.tan(math.radians(fovx_deg) / 2.0))
    return Camera(view=view.astype(np.float32), fx=float(np.float32(fx)), fy=float(np.float32(fx)),
                  cx=float(np.float32((width - 1) / 2.0)), cy=float(np.float32((height - 1) / 2.0)),
                  near=float(np.float32(near)), cam_pos=eye.astype(np.float32),
                  width=int(width), height=int(height))


def orbit_cameras(count=50, radius=4.0, width=1920, height=1080, fovx_deg=60.0):
    """`count` cameras at angle 2*pi*k/count on the circle of `radius` in y = 0, looking at 0."""
    cams = []
    for k in range(count):
        a = 2.0 * math.pi * k / count
        cams.append(look_at((radius * math.cos(a), 0.0, radius * math.sin(a)),
                            width=width, height=height, fovx_deg=fovx_deg))
    return cams


def sphere_camera(rng: np.random.Generator, radius=4.0, width=1280, height=720, fovx_deg=60.0):
    """Random camera on the sphere of `radius`, looking at the origin."""
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    return look_at(radius * v, width=width, height=height, fovx_deg=fovx_deg)


def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _random_rotations(rng, k):
    """k random 3x3 rotation matrices from the QR factorisation of Gaussian matrices."""
    out = np.empty((k, 3, 3))
    for i in range(k):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out[i] = q
    return out


def _attributes(rng, n, log_scale_mean=-4.0, log_scale_std=0.5):
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3)))
    rots = _unit_quats(rng, n)
    opac = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, size=n)))
    sh = rng.normal(0.0, 0.2, size=(n, 16, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    return scales, rots, opac, sh


def _pack(means, scales, rots, opac, sh) -> Scene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f(means), f(scales), f(rots), f(opac), f(sh))


def tiny_scene(seed=0, n=10_000) -> Scene:
    """Means U[-1,1]^3; log-scales N(-4, 0.5); random unit quaternions;
    opacity sigmoid(N(0, 1.5)); SH DC N(0.5, 0.2), higher bands N(0, 0.2)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    return _pack(means, *_attributes(rng, n))


def _cluster_means(rng, n, clusters=64):
    n_bg = n // 10
    n_cl = n - n_bg
    centres = rng.uniform(-3.0, 3.0, size=(clusters, 3))
    rot = _random_rotations(rng, clusters)
    stds = rng.uniform(0.1, 0.6, size=(clusters, 3))
    which = rng.integers(0, clusters, size=n_cl)
    local = rng.normal(size=(n_cl, 3)) * stds[which]
    pts = centres[which] + np.einsum("nij,nj->ni", rot[which], local)
    bg = rng.uniform(-10.0, 10.0, size=(n_bg, 3))
    means = np.concatenate([pts, bg])
    return means[rng.permutation(n)]


def cluster_scene(n=1_000_000, seed=1) -> Scene:
    """90% of means in 64 anisotropic clusters (centres U[-3,3]^3, random
    rotation, axis stds U[0.1, 0.6]) plus 10% uniform in [-10,10]^3."""
    rng = np.random.default_rng(seed)
    means = _cluster_means(rng, n)
    return _pack(means, *_attributes(rng, n))


def heavy_scene(n=3_000_000, seed=2, dense_fraction=0.3, dense_std=0.22) -> Scene:
    """Like `cluster_scene` but 30% of the Gaussians sit in one isotropic
    cluster (std 0.22) at the origin with log-scales N(-3, 0.7), giving highly
    uneven per-pixel loads (the paper's uneven-load setting, Sec. 4.4)."""
    rng = np.random.default_rng(seed)
    n_dense = int(n * dense_fraction)
    n_rest = n - n_dense
    rest_means = _cluster_means(rng, n_rest)
    rest = _attributes(rng, n_rest)
    dense_means = rng.normal(0.0, dense_std, size=(n_dense, 3))
    dense = _attributes(rng, n_dense, log_scale_mean=-3.0, log_scale_std=0.7)
    means = np.concatenate([rest_means, dense_means])
    attrs = [np.concatenate([a, b]) for a, b in zip(rest, dense)]
    perm = rng.permutation(n)
    return _pack(means[perm], *(a[perm] for a in attrs))


def deep_scene(n=20_000, seed=9, z_eye=-3.0, near=0.25, far=40_000.0) -> Scene:
    """Gaussians in front of a camera at (0, 0, z_eye) looking along +z, at
    view depths log-uniform in [near, far] (17 octaves), inside the 60-degree
    frustum, with scales proportional to the depth (a few pixels each).  The
    depth keys of the visible Gaussians then span more than 2^27."""
    rng = np.random.default_rng(seed)
    d = np.exp(rng.uniform(np.log(near), np.log(far), size=n))
    half = np.tan(np.radians(30.0))
    x = rng.uniform(-0.9, 0.9, size=n) * half * d
    y = rng.uniform(-0.9, 0.9, size=n) * half * d
    means = np.stack([x, y, z_eye + d], axis=1)
    scales, rots, opac, sh = _attributes(rng, n)
    scales = scales / np.exp(-4.0) * 0.004 * d[:, None]
    return _pack(means, scales, rots, opac, sh)


def perturbed_scene(scene: Scene, seed=4, mean_std=0.01, logit_std=0.3) -> Scene:
    """Training target: means + N(0, 0.01), opacity logits + N(0, 0.3)."""
    rng = np.random.default_rng(seed)
    means = scene.means.astype(np.float64) + rng.normal(0.0, mean_std, size=scene.means.shape)
    o = np.clip(scene.opac.astype(np.float64), 1e-6, 1 - 1e-6)
    logit = np.log(o / (1 - o)) + rng.normal(0.0, logit_std, size=o.shape)
    opac = 1.0 / (1.0 + np.exp(-logit))
    return _pack(means, scene.scales, scene.rots, opac, scene.sh)


def isolated_gaussian(mean, scale, quat, opacity, dc_rgb) -> Scene:
    """A one-Gaussian scene whose colour comes from the SH DC band only."""
    sh = np.zeros((1, 16, 3))
    sh[0, 0, :] = dc_rgb
    return _pack(np.asarray([mean]), np.asarray([scale]), np.asarray([quat]),
                 np.asarray([opacity]), sh)
