"""Pins of the gradient oracle (oracle/grad.py).

Its forward must equal the C oracle's (which is pinned against closed forms
and brute force), and its autograd gradient of L = <w, image> must equal
central finite differences of the C oracle's FP64 forward.  The load term's
gradient has no finite-difference counterpart (the load is a count): the
straight-through reading is checked against its definition, and the early-stop
reading against the slope of the count the C oracle renders as the opacities
of a stack of Gaussians rise."""
import numpy as np
import pytest

import oracle
from oracle import grad as og
from paper_2409_08669_gb300 import scenes as S

torch = pytest.importorskip("torch")


def _small_scene(seed=21, n=300):
    sc = S.tiny_scene(seed, n=n)
    sc.means[:] = (sc.means * 0.6).astype(np.float32)
    return sc


def test_real_sh_basis_matches_c_oracle():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(25, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = og.real_sh_basis(torch.tensor(d), 3).numpy()
    for i in range(d.shape[0]):
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[i, l * l + l + m] == pytest.approx(oracle.real_sh(l, m, d[i]), abs=1e-12)


@pytest.mark.parametrize("mode", [S.MODE_PLAIN, S.MODE_AABB])
def test_torch_forward_equals_c_oracle(mode):
    sc = _small_scene()
    cam = S.look_at((0.2, -0.1, -2.5), width=40, height=36)
    st = S.Settings(mode=mode, bg=(0.1, 0.0, 0.3))
    ref = oracle.render(sc, cam, st)
    img, T, load = og.render_torch(og.leaf_params(sc), cam, st)
    np.testing.assert_allclose(img.detach().numpy(), ref["img"], atol=1e-12)
    np.testing.assert_allclose(T.detach().numpy(), ref["t_final"], atol=1e-12)
    np.testing.assert_array_equal(load.detach().numpy(), ref["load"])


def _c_loss(arrays, cam, st, w):
    sc = og._ArrScene(arrays)
    out = oracle.render(sc, cam, st)
    return float((out["img"] * w).sum()), out


def test_autograd_matches_finite_differences_of_c_oracle():
    sc = _small_scene(seed=5, n=200)
    cam = S.look_at((0.1, 0.2, -2.4), width=40, height=32)
    st = S.Settings(mode=S.MODE_AABB)
    rng = np.random.default_rng(11)
    w = rng.normal(size=(3, cam.height, cam.width))
    grads, _, _ = og.gradients(sc, cam, st, w)
    base = tuple(np.asarray(a, np.float64).copy() for a in sc.arrays())
    _, ref = _c_loss(base, cam, st, w)
    tiles = ref["pre"]["tiles"]
    cand = np.nonzero(tiles > 0)[0]
    checked = 0
    for t_idx, (name, shape) in enumerate(zip(("means", "scales", "rots", "opac", "sh"),
                                              [a.shape for a in base])):
        for _ in range(8):
            g = int(rng.choice(cand))
            rest = tuple(int(rng.integers(0, s)) for s in shape[1:])
            idx = (g,) + rest
            if name == "sh" and idx[1] > 15:
                continue
            theta = base[t_idx][idx]
            h = 1e-6 * max(abs(theta), 1e-2)
            vals = []
            for sgn in (1, -1):
                arrs = [a.copy() for a in base]
                arrs[t_idx][idx] = theta + sgn * h
                Lv, out = _c_loss(tuple(arrs), cam, st, w)
                # skip if a discrete decision moved (pairs, loads, stop points)
                if (out["load"] != ref["load"]).any() or out["keys"].shape != ref["keys"].shape \
                        or (out["keys"] != ref["keys"]).any():
                    vals = None
                    break
                vals.append(Lv)
            if vals is None:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            ga = grads[t_idx][idx]
            assert ga == pytest.approx(fd, rel=1e-4, abs=1e-6 * max(1.0, abs(fd))), (name, idx, ga, fd)
            checked += 1
    assert checked >= 25


def test_load_term_straight_through_definition():
    """d<v, load>/d(sigma) = sum over blended pixels of v * d(alpha)/d(sigma)
    with alpha = sigma * exp(-q/2) below the 0.99 clamp."""
    sc = S.isolated_gaussian((0, 0, 0), (0.05, 0.04, 0.03), (1, 0, 0, 0), 0.4, (0.5, 0.5, 0.5))
    cam = S.look_at((0, 0, -3), width=24, height=24)
    st = S.Settings()
    v = np.random.default_rng(2).normal(size=(24, 24))
    grads, img, load = og.gradients(sc, cam, st, np.zeros((3, 24, 24)), dl_dload=v)
    ref = oracle.render(sc, cam, st)
    alpha = 1.0 - ref["t_final"]                     # one Gaussian: T = 1 - alpha where blended
    sigma = float(np.float32(0.4))
    expect = float((v * (load > 0) * alpha / sigma).sum())
    assert grads[3][0] == pytest.approx(expect, rel=1e-10)


def test_load_term_early_stop_reading_on_a_stack():
    """The early-stop reading (load_grad = 1) on a column of identical
    Gaussians in front of the camera: the centre pixel stops after l blends,
    and raising any blended Gaussian's opacity brings the stop forward, so
    d l / d sigma < 0 there (the straight-through reading gives > 0).  Its size:
    -l / (-ln T_final) * d(-ln(1 - alpha_k))/d sigma summed over the blended k."""
    k = 30
    means = np.zeros((k, 3)); means[:, 2] = np.linspace(-0.5, 0.5, k)
    sc = S.Scene(*(np.ascontiguousarray(a, dtype=np.float32) for a in (
        means, np.full((k, 3), 0.08), np.tile([1.0, 0.0, 0.0, 0.0], (k, 1)), np.full(k, 0.5),
        np.zeros((k, 16, 3)))))
    cam = S.look_at((0, 0, -3), width=17, height=17)
    v = np.zeros((17, 17)); v[8, 8] = 1.0
    out = {}
    for lg in (S.LOAD_GRAD_STRAIGHT, S.LOAD_GRAD_TERMINATION):
        st = S.Settings(mode=S.MODE_AABB, load_grad=lg)
        grads, img, load = og.gradients(sc, cam, st, np.zeros((3, 17, 17)), dl_dload=v)
        out[lg] = (grads[3], load)
    ref = oracle.render(sc, cam, S.Settings(mode=S.MODE_AABB))
    l = int(ref["load"][8, 8])
    assert 0 < l < k and ref["t_final"][8, 8] < 1e-3           # the centre pixel stopped early
    g_st, g_stop = out[S.LOAD_GRAD_STRAIGHT][0].sum(), out[S.LOAD_GRAD_TERMINATION][0].sum()
    assert g_st > 0 and g_stop < 0
    # magnitude: each blended Gaussian is centred on the pixel (on the optical
    # axis), so its alpha there is sigma itself and T_final = (1 - sigma)^l
    sigma = 0.5
    t_final = ref["t_final"][8, 8]
    assert t_final == pytest.approx((1.0 - sigma) ** l, rel=1e-9)
    expect = -l / -np.log(t_final) * l * (1.0 / (1.0 - sigma))   # d alpha/d sigma = 1
    assert g_stop == pytest.approx(expect, rel=1e-6)


def _stack(sigma, k=30):
    means = np.zeros((k, 3)); means[:, 2] = np.linspace(-0.5, 0.5, k)
    return S.Scene(*(np.ascontiguousarray(a, dtype=np.float32) for a in (
        means, np.full((k, 3), 0.08), np.tile([1.0, 0.0, 0.0, 0.0], (k, 1)), np.full(k, sigma),
        np.zeros((k, 16, 3)))))


def test_load_term_early_stop_reading_follows_the_slope_of_the_count():
    """Independent of the reading's formula: the C oracle's integer load at the
    centre pixel of the stack (all opacities equal to sigma) falls one step at
    a time as sigma sweeps [0.4, 0.6] (18 blends down to 10); the least-squares
    slope of that staircase is what a smooth d l / d sigma must match.  The
    early-stop reading, summed over the blended Gaussians at sigma = 0.5,
    agrees within 10% (measured: -37.5 against -39.1); the straight-through
    reading (+13, the count itself) has the wrong sign."""
    cam = S.look_at((0, 0, -3), width=17, height=17)
    sig = np.linspace(0.4, 0.6, 81)
    counts = np.array([oracle.render(_stack(s), cam, S.Settings(mode=S.MODE_AABB))["load"][8, 8]
                       for s in sig])
    assert counts[0] == 18 and counts[-1] == 10 and np.all(np.diff(counts) <= 0)
    slope = np.polyfit(sig, counts, 1)[0]
    v = np.zeros((17, 17)); v[8, 8] = 1.0
    got = {}
    for lg in (S.LOAD_GRAD_STRAIGHT, S.LOAD_GRAD_TERMINATION):
        st = S.Settings(mode=S.MODE_AABB, load_grad=lg)
        grads, _, _ = og.gradients(_stack(0.5), cam, st, np.zeros((3, 17, 17)), dl_dload=v)
        got[lg] = float(grads[3].sum())
    assert got[S.LOAD_GRAD_TERMINATION] == pytest.approx(slope, rel=0.10)
    assert got[S.LOAD_GRAD_STRAIGHT] > 0 > slope


def test_clamp_near_pixels_single_gaussian_on_a_pixel_centre():
    """One Gaussian centred exactly on pixel (32, 32) of a 65x65 image: its
    unclamped opacity there is sigma itself (q = 0), so with sigma = 0.99 the
    centre pixel is flagged and pixels where exp(-q/2) has fallen by more
    than the tolerance are not; with sigma = 0.5 the clamp is never near."""
    cam = S.look_at((0, 0, -3), width=65, height=65)
    assert cam.cx == 32.0 and cam.cy == 32.0
    for sigma, flagged in ((0.99, True), (0.5, False)):
        sc = S.isolated_gaussian((0, 0, 0), (0.05, 0.05, 0.05), (1, 0, 0, 0), sigma, (0.5, 0.5, 0.5))
        m = og.clamp_near_pixels(sc, cam, S.Settings(mode=S.MODE_AABB))
        assert bool(m[32, 32]) == flagged
        assert int(m.sum()) == (1 if flagged else 0)
