"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here compares the oracle with something other than itself:
closed forms derived by hand for special cases, a library routine (numpy
eigvalsh, scipy's spherical harmonics, numpy's stable sort), numerical
differentiation, brute-force sampling, or an invariant.  A plausible slip in
the oracle (a transposed rotation, a dropped Jacobian term, a wrong SH sign,
an off-by-one tile edge, a reordered blend) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2409_08669_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _single(mean, scale, quat, opacity, dc=(0.4, 0.6, 0.8)):
    return S.isolated_gaussian(mean, scale, quat, opacity, dc)


def _quat_z(theta):
    """Unit quaternion (w, x, y, z) of a rotation by theta about +z."""
    return (math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2))


def _f32(v):
    return float(np.float32(v))


def _theta_f32(theta):
    """Rotation angle actually encoded by the float32-rounded quaternion."""
    w, _, _, z = (np.float32(v) for v in _quat_z(theta))
    return 2.0 * math.atan2(float(z), float(w))


def _analytic_cov2d_centre(f, z0, s1, s2, theta, lowpass=0.3):
    """Sigma' of a Gaussian at the world origin seen by look_at((0,0,-z0)).

    The camera frame is world rotated by pi about z, which commutes with the
    Gaussian's rotation about z, and at the optical axis J = diag(f/z0, f/z0),
    so Sigma' = (f/z0)^2 R(theta) diag(s1^2, s2^2) R(theta)^T + lowpass I."""
    c, s = math.cos(theta), math.sin(theta)
    k = (f / z0) ** 2
    a = k * (c * c * s1 * s1 + s * s * s2 * s2) + lowpass
    b = k * c * s * (s1 * s1 - s2 * s2)
    cc = k * (s * s * s1 * s1 + c * c * s2 * s2) + lowpass
    return a, b, cc


# ----------------------------------------------------------------------------
# Paper constants
# ----------------------------------------------------------------------------

def test_settings_defaults_match_paper_constants():
    g = json.load(open(GOLDEN))
    st = S.Settings()
    assert st.alpha_low == pytest.approx(1.0 / 255.0, rel=1e-7)
    assert g["alpha_low"]["value"] == "1/255"
    assert oracle.TILE == g["tile_size"]["value"] == 16


# ----------------------------------------------------------------------------
# Projection: rotation convention, Jacobian, clamp, pixel centre (Sec. 3.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1, -0.7, 2.5])
def test_cov2d_closed_form_at_centre(theta):
    z0, s1, s2, s3 = 3.0, 0.05, 0.02, 0.01
    cam = S.look_at((0, 0, -z0), width=128, height=96)
    sc = _single((0, 0, 0), (s1, s2, s3), _quat_z(theta), 0.3)
    pre = oracle.preprocess(sc, cam, S.Settings())
    g = pre["geom"][0]
    a, b, c = _analytic_cov2d_centre(cam.fx, z0, _f32(s1), _f32(s2), _theta_f32(theta),
                                     lowpass=_f32(0.3))
    assert g[oracle.G_COV_A] == pytest.approx(a, rel=1e-6)
    assert g[oracle.G_COV_B] == pytest.approx(b, rel=1e-6, abs=1e-9)
    assert g[oracle.G_COV_C] == pytest.approx(c, rel=1e-6)
    assert g[oracle.G_PX] == pytest.approx(cam.cx, abs=1e-9)
    assert g[oracle.G_PY] == pytest.approx(cam.cy, abs=1e-9)
    # conic is the inverse
    M = np.array([[a, b], [b, c]])
    Minv = np.linalg.inv(M)
    assert g[oracle.G_CONIC_A] == pytest.approx(Minv[0, 0], rel=1e-6)
    assert g[oracle.G_CONIC_B] == pytest.approx(Minv[0, 1], rel=1e-6, abs=1e-12)
    assert g[oracle.G_CONIC_C] == pytest.approx(Minv[1, 1], rel=1e-6)


def _proj(cam, p):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


@pytest.mark.parametrize("mean", [(0.4, -0.3, 0.5), (-0.6, 0.2, -0.4), (0.1, 0.5, 1.0)])
def test_cov2d_matches_numerical_jacobian(mean):
    """Off-axis: Sigma' = J Sigma_cam J^T + 0.3 I with J from central differences."""
    cam = S.look_at((0.3, 0.2, -3.0), target=(0.1, 0, 0), width=200, height=160)
    q = np.array([0.8, 0.3, -0.4, 0.2]); q /= np.linalg.norm(q)
    scale = np.array([0.07, 0.03, 0.05])
    sc = _single(mean, scale, q, 0.3)
    pre = oracle.preprocess(sc, cam, S.Settings())
    g = pre["geom"][0]
    V = cam.view.astype(np.float64)
    # use the float32 values both sides actually receive
    mean = sc.means[0].astype(np.float64)
    q = sc.rots[0].astype(np.float64); q /= np.linalg.norm(q)
    scale = sc.scales[0].astype(np.float64)
    p = V[:3, :3] @ mean + V[:3, 3]
    h = 1e-5
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = h
        J[:, k] = (_proj(cam, p + e) - _proj(cam, p - e)) / (2 * h)
    # rotation from the quaternion via scipy-free Rodrigues: axis-angle
    w, x, y, z = q
    ang = 2 * math.acos(w)
    axis = np.array([x, y, z]) / math.sin(ang / 2)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    Sig = R @ np.diag(scale ** 2) @ R.T
    Sc = V[:3, :3] @ Sig @ V[:3, :3].T
    C2 = J @ Sc @ J.T + _f32(0.3) * np.eye(2)
    assert g[oracle.G_COV_A] == pytest.approx(C2[0, 0], rel=2e-6)
    assert g[oracle.G_COV_B] == pytest.approx(C2[0, 1], rel=2e-6, abs=1e-6)
    assert g[oracle.G_COV_C] == pytest.approx(C2[1, 1], rel=2e-6)
    px = _proj(cam, p)
    assert g[oracle.G_PX] == pytest.approx(px[0], abs=1e-9)
    assert g[oracle.G_PY] == pytest.approx(px[1], abs=1e-9)


def test_jacobian_clamp_freezes_offaxis_term():
    """Beyond +-1.3 tan(fov/2) the Jacobian uses the clamped x/z, so moving the
    Gaussian further out (same depth, isotropic) leaves Sigma' unchanged."""
    cam = S.look_at((0, 0, -3), width=100, height=100)
    st = S.Settings()
    out = []
    for x in (-3.0, -4.0):  # world x -> camera -x; z_cam = 3; limit 1.3*tan(30deg)*3 = 2.25
        sc = _single((x, 0.0, 0.0), (0.05, 0.05, 0.05), (1, 0, 0, 0), 0.5)
        out.append(oracle.preprocess(sc, cam, st)["geom"][0, oracle.G_COV_A:oracle.G_COV_C + 1])
    np.testing.assert_allclose(out[0], out[1], rtol=1e-12)
    sc = _single((-2.0, 0.0, 0.0), (0.05, 0.05, 0.05), (1, 0, 0, 0), 0.5)  # inside the clamp
    inside = oracle.preprocess(sc, cam, st)["geom"][0, oracle.G_COV_A]
    assert abs(inside - out[0][0]) > 1e-3


def test_near_plane_cull_and_depth_bits():
    cam = S.look_at((0, 0, -3), width=64, height=64)
    sc = _single((0, 0, -2.85), (0.01, 0.01, 0.01), (1, 0, 0, 0), 0.9)  # depth 0.15 < 0.2
    pre = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_PLAIN))
    assert pre["flags"][0] & oracle.F_VISIBLE == 0 and pre["tiles"][0] == 0
    sc = _single((0.1, -0.2, 0.5), (0.01, 0.01, 0.01), (1, 0, 0, 0), 0.9)
    pre = oracle.preprocess(sc, cam, S.Settings())
    v = cam.view.astype(np.float32)
    m = sc.means[0]
    d = np.float32(v[2, 0] * m[0])
    d = np.float32(d + np.float32(v[2, 1] * m[1]))
    d = np.float32(d + np.float32(v[2, 2] * m[2]))
    d = np.float32(d + v[2, 3])
    assert pre["depth"][0].view(np.uint32) == d.view(np.uint32)
    assert pre["geom"][0, oracle.G_VZ] == pytest.approx(3.5, abs=1e-6)


# ----------------------------------------------------------------------------
# Radii: Eq. 5-8 (adaptive radius) and Eq. 9-11 (AABB)
# ----------------------------------------------------------------------------

def _boundary_extremes(cov, L, n=20000):
    """Sample the ellipse x^T cov^{-1} x = 2L (Eq. 5) by angle; return the
    largest distance, largest |x| and largest |y| on it."""
    th = np.linspace(0, 2 * np.pi, n, endpoint=False)
    u = np.stack([np.cos(th), np.sin(th)])
    inv = np.linalg.inv(cov)
    rho = np.sqrt(2 * L / np.einsum("in,ij,jn->n", u, inv, u))
    pts = u * rho
    return rho.max(), np.abs(pts[0]).max(), np.abs(pts[1]).max()


def _random_gaussians(rng, k, opac_hi=0.3):
    out = []
    for _ in range(k):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        s = np.exp(rng.normal(-3.5, 0.6, size=3))
        m = rng.uniform(-0.5, 0.5, size=3)
        out.append((m, s, q, rng.uniform(0.01, opac_hi)))
    return out


@pytest.mark.parametrize("alpha_low", [float(np.float32(1 / 255)), float(np.float32(4 / 255))],
                         ids=["1/255", "4/255"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adaptive_radius_and_aabb_against_sampled_ellipse(seed, alpha_low):
    rng = np.random.default_rng(seed)
    cam = S.look_at((0, 0, -3), width=256, height=256)
    for m, s, q, op in _random_gaussians(rng, 20):
        sc = _single(m, s, q, op)
        circ = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_CIRCLE, alpha_low=alpha_low))["geom"][0]
        aabb = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_AABB, alpha_low=alpha_low))["geom"][0]
        cov = np.array([[circ[oracle.G_COV_A], circ[oracle.G_COV_B]],
                        [circ[oracle.G_COV_B], circ[oracle.G_COV_C]]])
        L = math.log(float(np.float32(op)) / alpha_low)
        if L <= 0:   # sigma <= alpha_low: no real radius, no pairs
            assert circ[oracle.G_RX] == 0 and aabb[oracle.G_RX] == 0
            continue
        rmax, xmax, ymax = _boundary_extremes(cov, L)
        # sigma <= 0.3 < alpha_low * e^4.5, so the r_o cap does not bind
        assert circ[oracle.G_RX] < circ[oracle.G_RO]
        assert circ[oracle.G_RX] == pytest.approx(rmax, rel=1e-6)
        assert aabb[oracle.G_RX] == pytest.approx(xmax, rel=1e-6)
        assert aabb[oracle.G_RY] == pytest.approx(ymax, rel=1e-6)
        # larger eigenvalue and r_o = ceil(3 sqrt(lambda'_max))
        lam = np.linalg.eigvalsh(cov)[-1]
        assert circ[oracle.G_LAMBDA] == pytest.approx(lam, rel=1e-12)
        assert circ[oracle.G_RO] == math.ceil(3 * math.sqrt(lam))
        # Eq. 6 coefficients: r_ad = sqrt(2D / (-(A+B) + sqrt((A-B)^2 + C^2)))
        A, B, C = cov[1, 1], cov[0, 0], -2 * cov[0, 1]
        D = -2 * (cov[0, 0] * cov[1, 1] - cov[0, 1] ** 2) * L
        r_abcd = math.sqrt(2 * D / (-(A + B) + math.sqrt((A - B) ** 2 + C ** 2)))
        assert circ[oracle.G_RX] == pytest.approx(r_abcd, rel=1e-9)
        # invariants: max(x_max, y_max) <= r_ad <= hypot(x_max, y_max)
        r_ad, xm, ym = circ[oracle.G_RX], aabb[oracle.G_RX], aabb[oracle.G_RY]
        assert max(xm, ym) <= r_ad * (1 + 1e-12)
        assert r_ad <= math.hypot(xm, ym) * (1 + 1e-12)


def test_axis_aligned_cov_gives_r_ad_equal_larger_half_axis():
    cam = S.look_at((0, 0, -3), width=256, height=256)
    sc = _single((0, 0, 0), (0.06, 0.02, 0.02), (1, 0, 0, 0), 0.2)  # theta = 0: axis aligned
    c = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_CIRCLE))["geom"][0]
    a = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_AABB))["geom"][0]
    assert abs(c[oracle.G_COV_B]) < 1e-12
    assert c[oracle.G_RX] == pytest.approx(max(a[oracle.G_RX], a[oracle.G_RY]), rel=1e-12)


def test_opacity_below_alpha_low_emits_no_pairs_in_adaptive_modes():
    cam = S.look_at((0, 0, -3), width=64, height=64)
    sc = _single((0, 0, 0), (0.05, 0.05, 0.05), (1, 0, 0, 0), 0.003)  # < 1/255
    for mode, expect_pairs in ((S.MODE_PLAIN, True), (S.MODE_CIRCLE, False), (S.MODE_AABB, False)):
        pre = oracle.preprocess(sc, cam, S.Settings(mode=mode))
        assert (pre["tiles"][0] > 0) == expect_pairs
        out = oracle.render(sc, cam, S.Settings(mode=mode))
        assert out["img"].max() == 0.0 and out["load"].max() == 0


def test_rcap_binds_for_opaque_gaussians():
    """r_ad < r_o  iff  sigma < alpha_low e^{4.5} (up to the ceil of r_o)."""
    cam = S.look_at((0, 0, -3), width=256, height=256)
    for op, capped in ((0.9, True), (0.2, False)):
        sc = _single((0, 0, 0), (0.05, 0.03, 0.02), _quat_z(0.4), op)
        g = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_CIRCLE))["geom"][0]
        assert (g[oracle.G_RX] == g[oracle.G_RO]) == capped


# ----------------------------------------------------------------------------
# Tile rule: pairs are exactly the tiles holding a pixel centre inside the box
# ----------------------------------------------------------------------------

def _brute_tiles(px, py, rx, ry, w, h):
    xs = np.arange(w); ys = np.arange(h)
    inx = np.abs(xs - px) <= rx
    iny = np.abs(ys - py) <= ry
    tiles = set()
    for y in ys[iny]:
        for x in xs[inx]:
            tiles.add((y // 16) * ((w + 15) // 16) + x // 16)
    return tiles


@pytest.mark.parametrize("seed", [3, 4])
def test_pair_tiles_equal_pixel_brute_force(seed):
    rng = np.random.default_rng(seed)
    w, h = 150, 120  # ragged last tile row and column
    cam = S.look_at((0, 0, -2.5), width=w, height=h)
    for m, s, q, op in _random_gaussians(rng, 25, opac_hi=0.99):
        sc = _single(m * 2.0, s * 2.0, q, op)
        for mode in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB):
            pre = oracle.preprocess(sc, cam, S.Settings(mode=mode))
            keys, vals = oracle.emit_pairs(pre)
            got = set((keys >> np.uint64(32)).astype(np.int64).tolist())
            g = pre["geom"][0]
            if pre["tiles"][0] == 0 and g[oracle.G_RX] == 0:
                assert not got
                continue
            want = _brute_tiles(g[oracle.G_PX], g[oracle.G_PY], g[oracle.G_RX], g[oracle.G_RY], w, h)
            assert got == want


def _brute_tiles_3dgs(px, py, rx, ry, w, h):
    """The 3DGS rounding as a point set: with R = ceil(r), the tiles whose span
    [16t, 16t + 16) meets the real interval [c - R, c + R - 1], kept inside the
    tile grid.  Sampled every half pixel plus both ends (tiles are 16 wide)."""
    def axis(c, r, size):
        R = math.ceil(r)
        lo, hi = c - R, c + R - 1
        if hi < lo:
            return set()
        pts = np.append(np.arange(lo, hi, 0.5), hi)
        t = set(np.floor(pts / 16).astype(np.int64).tolist())
        return {v for v in t if 0 <= v < (size + 15) // 16}
    tx, ty = axis(px, rx, w), axis(py, ry, h)
    return {y * ((w + 15) // 16) + x for y in ty for x in tx}


@pytest.mark.parametrize("seed", [3, 5])
def test_3dgs_rect_rule_equals_point_set_brute_force(seed):
    rng = np.random.default_rng(seed)
    w, h = 150, 120
    cam = S.look_at((0, 0, -2.5), width=w, height=h)
    n_checked = 0
    for m, s, q, op in _random_gaussians(rng, 25, opac_hi=0.99):
        sc = _single(m * 2.0, s * 2.0, q, op)
        for mode in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB):
            pre = oracle.preprocess(sc, cam, S.Settings(mode=mode, rect_rule=S.RECT_3DGS))
            keys, _ = oracle.emit_pairs(pre)
            got = set((keys >> np.uint64(32)).astype(np.int64).tolist()) if pre["tiles"][0] else set()
            g = pre["geom"][0]
            if not (pre["flags"][0] & oracle.F_VISIBLE) or g[oracle.G_RX] == 0:
                assert not got
                continue
            want = _brute_tiles_3dgs(g[oracle.G_PX], g[oracle.G_PY], g[oracle.G_RX], g[oracle.G_RY], w, h)
            assert got == want
            n_checked += 1
    assert n_checked > 30


def test_3dgs_rect_rule_drops_edge_tiles_and_is_not_lossless():
    """The 3DGS rounding keeps the lower tiles of the pixel rule (or one more)
    and loses the last tile when px + R falls in [16k, 16k + 1): the pixel 16k
    is then within the radius but its tile is not listed, so the image can
    differ from the lossless render, which equals the per-pixel brute force."""
    sc = S.tiny_scene(0, n=4000)
    cam = S.look_at((0, 0, -3), width=128, height=128)
    pix = oracle.render(sc, cam, S.Settings(mode=S.MODE_PLAIN))
    cmp = oracle.render(sc, cam, S.Settings(mode=S.MODE_PLAIN, rect_rule=S.RECT_3DGS))
    rp, rc = pix["pre"]["rect"], cmp["pre"]["rect"]
    both = (pix["pre"]["tiles"] > 0) & (cmp["pre"]["tiles"] > 0)
    assert np.all(rc[both, 0] <= rp[both, 0]) and np.all(rc[both, 1] <= rp[both, 1])
    assert np.all(rc[both, 2] >= rp[both, 2] - 1) and np.all(rc[both, 3] >= rp[both, 3] - 1)
    g = pix["pre"]["geom"]
    upper = np.floor(g[:, oracle.G_PX] + g[:, oracle.G_RO])
    dropped_x = both & (rc[:, 2] == rp[:, 2] - 1)
    # exactly the predicted edge case (inside the image) drops a column of tiles
    assert np.all(np.mod(upper[dropped_x], 16) == 0)
    assert dropped_x.sum() > 0
    assert np.abs(cmp["img"] - pix["img"]).max() > 1e-3
    # the compat render is still the render of its own tile lists
    bf = oracle.render_brute(cmp["pre"], S.Settings(mode=S.MODE_PLAIN), use_rect=True)
    np.testing.assert_array_equal(cmp["img"], bf["img"])


# ----------------------------------------------------------------------------
# Colour: real SH basis (Condon-Shortley phase) vs scipy
# ----------------------------------------------------------------------------

def _scipy_real_sh(l, m, d):
    from scipy.special import sph_harm_y
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    if m == 0:
        return float(np.real(sph_harm_y(l, 0, theta, phi)))
    y = sph_harm_y(l, abs(m), theta, phi)  # includes the Condon-Shortley phase
    return float(math.sqrt(2) * (np.real(y) if m > 0 else np.imag(y)))


def test_real_sh_matches_scipy():
    rng = np.random.default_rng(7)
    for _ in range(40):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert oracle.real_sh(l, m, d) == pytest.approx(_scipy_real_sh(l, m, d), abs=1e-12)


def test_real_sh_orthonormal_by_quadrature():
    n_t, n_p = 64, 128
    xg, wg = np.polynomial.legendre.leggauss(n_t)  # cos(theta) nodes
    phis = np.arange(n_p) * 2 * np.pi / n_p
    basis = []
    for l in range(4):
        for m in range(-l, l + 1):
            vals = np.empty((n_t, n_p))
            for i, t in enumerate(xg):
                st = math.sqrt(1 - t * t)
                for j, p in enumerate(phis):
                    vals[i, j] = oracle.real_sh(l, m, (st * math.cos(p), st * math.sin(p), t))
            basis.append(vals)
    B = np.stack(basis)  # [16, n_t, n_p]
    W = wg[:, None] * (2 * np.pi / n_p)
    G = np.einsum("aij,bij,ij->ab", B, B, W)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-10)


def test_dc_colour_of_isolated_gaussian():
    cam = S.look_at((0, 0, -3), width=32, height=32)
    dc = (0.4, -0.9, 1.5)
    sc = _single((0, 0, 0), (0.02, 0.02, 0.02), (1, 0, 0, 0), 0.5, dc=dc)
    rgb = oracle.preprocess(sc, cam, S.Settings())["rgb"][0]
    y00 = 0.5 / math.sqrt(math.pi)
    expect = [max(0.0, float(np.float32(v)) * y00 + 0.5) for v in dc]
    np.testing.assert_allclose(rgb, expect, rtol=1e-12)


# ----------------------------------------------------------------------------
# Blending: single-Gaussian footprint and hand-worked stacks (Eq. 2-3, 12)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("theta,op", [(0.0, 0.3), (0.7, 0.9), (-1.2, 0.05)])
def test_single_gaussian_image_closed_form(theta, op):
    z0, s1, s2 = 3.0, 0.04, 0.015
    w, h = 96, 80
    cam = S.look_at((0, 0, -z0), width=w, height=h)
    dc = (0.9, 0.2, 0.5)
    sc = _single((0, 0, 0), (s1, s2, 0.01), _quat_z(theta), op, dc=dc)
    st = S.Settings(mode=S.MODE_AABB)
    out = oracle.render(sc, cam, st)
    a, b, c = _analytic_cov2d_centre(cam.fx, z0, _f32(s1), _f32(s2), _theta_f32(theta),
                                     lowpass=_f32(0.3))
    inv = np.linalg.inv(np.array([[a, b], [b, c]]))
    X, Y = np.meshgrid(np.arange(w) - cam.cx, np.arange(h) - cam.cy)
    q = inv[0, 0] * X * X + 2 * inv[0, 1] * X * Y + inv[1, 1] * Y * Y
    sigma = float(np.float32(op))
    alpha = np.minimum(0.99, sigma * np.exp(-0.5 * q))
    keep = alpha >= st.alpha_low
    # the r_o square can clip an opaque Gaussian's footprint
    r_o = math.ceil(3 * math.sqrt(np.linalg.eigvalsh(np.array([[a, b], [b, c]]))[-1]))
    tiles_x = [(int(math.ceil(cam.cx - r_o)) // 16), int(math.floor(cam.cx + r_o)) // 16]
    tiles_y = [(int(math.ceil(cam.cy - r_o)) // 16), int(math.floor(cam.cy + r_o)) // 16]
    xs, ys = np.meshgrid(np.arange(w) // 16, np.arange(h) // 16)
    in_tiles = (xs >= max(tiles_x[0], 0)) & (xs <= tiles_x[1]) & (ys >= max(tiles_y[0], 0)) & (ys <= tiles_y[1])
    keep &= in_tiles
    y00 = 0.5 / math.sqrt(math.pi)
    rgb = np.array([max(0.0, float(np.float32(v)) * y00 + 0.5) for v in dc])
    expect = rgb[:, None, None] * np.where(keep, alpha, 0.0)[None]
    np.testing.assert_allclose(out["img"], expect, atol=1e-12)
    np.testing.assert_allclose(out["t_final"], np.where(keep, 1 - alpha, 1.0), atol=1e-12)
    np.testing.assert_array_equal(out["load"], keep.astype(np.int32))


def test_two_gaussian_stack_worked_example():
    """Two Gaussians centred on the same pixel: at that pixel q = 0, alpha =
    sigma, and Eq. 3 gives C = c_front a_f + c_back a_b (1 - a_f)."""
    cam = S.look_at((0, 0, -3), width=16, height=16)
    front = (0.5, 0.5, 0.0)  # world -> camera flips x, y; centre pixel (7.5, 7.5) offset by fx*...
    # place both on the optical axis so they project to (cx, cy) = (7.5, 7.5);
    # evaluate at pixel (7, 7): q from the analytic isotropic Sigma'
    s = 0.01
    sc_f = _single((0, 0, -0.5), (s, s, s), (1, 0, 0, 0), 0.6, dc=(1.0, 0.0, 0.0))
    sc_b = _single((0, 0, 0.5), (s, s, s), (1, 0, 0, 0), 0.7, dc=(0.0, 1.0, 0.0))
    sc = S.Scene(*(np.concatenate([a, b]) for a, b in zip(sc_b.arrays(), sc_f.arrays())))
    out = oracle.render(sc, cam, S.Settings())
    y00 = 0.5 / math.sqrt(math.pi)
    cf = np.array([1.0 * y00 + 0.5, 0.5, 0.5])
    cb = np.array([0.5, 1.0 * y00 + 0.5, 0.5])
    dx = dy = 0.5  # pixel (7, 7) to centre (7.5, 7.5)
    def alpha(z_cam, op):
        var = (cam.fx * _f32(s) / z_cam) ** 2 + _f32(0.3)
        return min(0.99, float(np.float32(op)) * math.exp(-0.5 * (dx * dx + dy * dy) / var))
    af, ab = alpha(2.5, 0.6), alpha(3.5, 0.7)
    expect = cf * af + cb * ab * (1 - af)
    np.testing.assert_allclose(out["img"][:, 7, 7], expect, atol=1e-12)
    assert out["t_final"][7, 7] == pytest.approx((1 - af) * (1 - ab), abs=1e-12)
    assert out["load"][7, 7] == 2
    del front


def test_early_termination_worked_example():
    """Three opaque (alpha clamped to 0.99) Gaussians at one pixel: T goes
    1 -> 0.01 -> 1e-4 (kept, since 1e-4 >= float32(1e-4)), and the third would
    give 1e-6 < t_min, so it is neither blended nor counted."""
    cam = S.look_at((0, 0, -3), width=16, height=16)
    gs = [_single((0, 0, z), (3.0, 3.0, 3.0), (1, 0, 0, 0), 0.999, dc=(c, c, c))
          for z, c in ((-1.0, 1.0), (0.0, 0.0), (1.0, -1.0))]
    sc = S.Scene(*(np.concatenate(x) for x in zip(*(g.arrays() for g in gs))))
    out = oracle.render(sc, cam, S.Settings())
    y00 = 0.5 / math.sqrt(math.pi)
    c1, c2 = 1.0 * y00 + 0.5, 0.5
    expect = c1 * 0.99 + c2 * 0.99 * (1 - 0.99)
    # pixel (7, 7) is 0.5 px from the centre; the huge Sigma' keeps alpha clamped
    assert out["img"][0, 7, 7] == pytest.approx(expect, abs=1e-12)
    assert out["load"][7, 7] == 2
    assert out["t_final"][7, 7] == pytest.approx((1 - 0.99) ** 2, rel=1e-12)


# ----------------------------------------------------------------------------
# Sort and ranges: numpy's stable sort and searchsorted
# ----------------------------------------------------------------------------

def test_sort_and_ranges_against_numpy():
    sc = S.tiny_scene(0, n=3000)
    cam = S.look_at((0, 0, -3), width=200, height=136)
    pre = oracle.preprocess(sc, cam, S.Settings())
    keys, vals = oracle.emit_pairs(pre)
    # emission is in Gaussian index order
    assert np.all(np.diff(vals.astype(np.int64)) >= 0)
    skeys, svals = oracle.sort_pairs(keys, vals)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(skeys, keys[order])
    np.testing.assert_array_equal(svals, vals[order])
    ranges = oracle.tile_ranges(skeys, cam.width, cam.height)
    tiles = (skeys >> np.uint64(32)).astype(np.int64)
    nt = ranges.shape[0]
    lo = np.searchsorted(tiles, np.arange(nt), side="left")
    hi = np.searchsorted(tiles, np.arange(nt), side="right")
    empty = lo == hi
    np.testing.assert_array_equal(ranges[~empty, 0], lo[~empty])
    np.testing.assert_array_equal(ranges[~empty, 1], hi[~empty])
    assert np.all(ranges[empty] == 0)
    assert int((ranges[:, 1] - ranges[:, 0]).sum()) == skeys.shape[0]


def test_sort_ties_keep_index_order():
    """Gaussians at one position share their depth bits, so their pairs have
    equal keys; the stable sort (Sec. 3.2, over index-order emission) keeps
    them in index order, as numpy's stable argsort does."""
    base = S.tiny_scene(1, n=40)
    idx = np.repeat(np.arange(8), 5)            # 8 positions, 5 Gaussians each
    sc = base.subset(np.arange(40))
    sc.means[:] = base.means[idx]
    cam = S.look_at((0.3, -0.2, -3), width=96, height=80)
    pre = oracle.preprocess(sc, cam, S.Settings(mode=S.MODE_PLAIN))
    keys, vals = oracle.emit_pairs(pre)
    skeys, svals = oracle.sort_pairs(keys, vals)
    assert np.unique(skeys).size < skeys.size   # ties present
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(svals, vals[order])


def test_depth_bits_follow_the_fixed_float32_order():
    """The sort depth is ((v20 x + v21 y) + v22 z) + v23 in float32, each
    product and sum rounded, in that order, for any camera orientation."""
    rng = np.random.default_rng(8)
    sc = S.tiny_scene(2, n=400)
    for _ in range(4):
        eye = rng.normal(size=3)
        eye = 3.0 * eye / np.linalg.norm(eye)
        cam = S.look_at(tuple(eye), width=64, height=48)
        pre = oracle.preprocess(sc, cam, S.Settings())
        v = cam.view.astype(np.float32)
        x, y, z = (sc.means[:, k].astype(np.float32) for k in range(3))
        d = v[2, 0] * x
        d = (d + v[2, 1] * y).astype(np.float32)
        d = (d + v[2, 2] * z).astype(np.float32)
        d = (d + v[2, 3]).astype(np.float32)
        np.testing.assert_array_equal(pre["depth"].view(np.uint32), d.view(np.uint32))


# ----------------------------------------------------------------------------
# Brute force, losslessness and nested culling (Sec. 4.2-4.3, Sec. 5.4)
# ----------------------------------------------------------------------------

def test_tiled_equals_brute_force_when_ro_does_not_bind():
    sc = S.tiny_scene(3, n=1500)
    sc.opac[:] = (sc.opac * 0.35).astype(np.float32)  # sigma < alpha_low e^4.5: r_ad <= r_o
    cam = S.look_at((0, 0, -3), width=64, height=64)
    for mode in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB):
        st = S.Settings(mode=mode)
        out = oracle.render(sc, cam, st)
        bf = oracle.render_brute(out["pre"], st)
        np.testing.assert_array_equal(out["img"], bf["img"])
        np.testing.assert_array_equal(out["load"], bf["load"])
        np.testing.assert_array_equal(out["t_final"], bf["t_final"])


def test_tiled_equals_brute_force_at_alpha_low_4_255_in_every_mode():
    """At alpha_low = 4/255 > e^-4.5 the 3-sigma radius r_o never binds: a
    pixel outside it has q > 9, so alpha <= sigma e^-4.5 < 4/255 for any
    sigma <= 1.  The tiled render (every mode, opacities up to 1) must then
    equal the per-pixel brute force over all Gaussians, with no tiles."""
    a4 = float(np.float32(4 / 255))
    assert a4 > math.exp(-4.5)
    sc = S.tiny_scene(6, n=1500)
    assert sc.opac.max() > 0.9
    cam = S.look_at((0.1, 0, -2.8), width=72, height=56)
    for mode in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB):
        st = S.Settings(mode=mode, alpha_low=a4)
        out = oracle.render(sc, cam, st)
        bf = oracle.render_brute(out["pre"], st)
        np.testing.assert_array_equal(out["img"], bf["img"])
        np.testing.assert_array_equal(out["load"], bf["load"])


def test_tiled_equals_rect_brute_force_general_scene():
    sc = S.tiny_scene(5, n=2000)
    cam = S.look_at((0, 0, -3), width=80, height=72)
    for mode in (S.MODE_PLAIN, S.MODE_AABB):
        st = S.Settings(mode=mode)
        out = oracle.render(sc, cam, st)
        bf = oracle.render_brute(out["pre"], st, use_rect=True)
        np.testing.assert_array_equal(out["img"], bf["img"])
        np.testing.assert_array_equal(out["load"], bf["load"])


def test_losslessness_and_nesting_on_tiny_scene():
    sc = S.tiny_scene(0, n=4000)
    cam = S.look_at((0, 0, -3), width=128, height=128)
    outs = {m: oracle.render(sc, cam, S.Settings(mode=m))
            for m in (S.MODE_PLAIN, S.MODE_CIRCLE, S.MODE_AABB)}
    base = outs[S.MODE_PLAIN]
    for m in (S.MODE_CIRCLE, S.MODE_AABB):
        np.testing.assert_array_equal(outs[m]["img"], base["img"])
        np.testing.assert_array_equal(outs[m]["load"], base["load"])
    # rectangles nest: AABB within CIRCLE within PLAIN, per Gaussian
    r = {m: outs[m]["pre"]["rect"] for m in outs}
    t = {m: outs[m]["pre"]["tiles"] for m in outs}
    for inner, outer in ((S.MODE_AABB, S.MODE_CIRCLE), (S.MODE_CIRCLE, S.MODE_PLAIN)):
        has = t[inner] > 0
        assert np.all(t[inner] <= t[outer])
        assert np.all(r[inner][has, 0] >= r[outer][has, 0]) and np.all(r[inner][has, 1] >= r[outer][has, 1])
        assert np.all(r[inner][has, 2] <= r[outer][has, 2]) and np.all(r[inner][has, 3] <= r[outer][has, 3])
    assert t[S.MODE_AABB].sum() < t[S.MODE_CIRCLE].sum() < t[S.MODE_PLAIN].sum()


def test_load_std_population_form():
    load = np.array([[0, 2], [4, 6]], np.int32)
    assert oracle.load_std(load) == pytest.approx(np.std(load.astype(np.float64)), rel=1e-15)
    assert oracle.load_std(np.full((3, 5), 7, np.int32)) == 0.0


# ----------------------------------------------------------------------------
# Planted mistakes: each pin above must catch a perturbed oracle.  These run
# the pins' checks against deliberately wrong stand-ins on the CPU.
# ----------------------------------------------------------------------------

def test_cov_pin_catches_transposed_rotation():
    theta = 0.6
    a, b, c = _analytic_cov2d_centre(500.0, 3.0, 0.05, 0.02, theta)
    a2, b2, c2 = _analytic_cov2d_centre(500.0, 3.0, 0.05, 0.02, -theta)  # R^T
    assert abs(b - b2) > 1e-3 * abs(b)


def test_sh_pin_catches_missing_condon_shortley_phase():
    d = np.array([0.3, -0.5, 0.81]); d /= np.linalg.norm(d)
    assert abs(oracle.real_sh(1, 1, d) + _scipy_real_sh(1, 1, d)) > 1e-3  # sign would flip
