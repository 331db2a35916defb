"""Planted mistakes in the oracle (CPU only).

Each case makes a copy of the oracle with one plausible error -- a dropped
term, a wrong sign or index, a swapped axis, a transposed operand, a
condition moved -- puts it in place of the real one and checks that one of
the pins fails: the C forward path (oracle/adr_oracle.c, compiled with gcc,
pins in test_oracle_pins.py) and the image loss (oracle/ssim.py, pins in
test_ssim_oracle.py).  The pin is first run on the real oracle, where it must
pass.  The gradient oracle (oracle/grad.py, pins in test_grad_oracle.py) is
treated the same way.  A site string that no longer occurs in the source
fails the test, so the cases follow edits of the oracle."""
import importlib.util
import os

import pytest

import oracle
from paper_2409_08669_gb300 import scenes as S
import test_grad_oracle as grad_pins
import test_oracle_pins as pins
import test_ssim_oracle as ssim_pins
from oracle import grad as ograd
from oracle import ssim as ossim

SRC = os.path.join(os.path.dirname(oracle.__file__), "adr_oracle.c")
A1 = S.Settings().alpha_low   # the paper's 1/255

# (name, text in adr_oracle.c, replacement, the pin that must catch it)
MUTANTS = [
    ("rotation_sign", "R[0][1] = 2 * (x * y - w * z);", "R[0][1] = 2 * (x * y + w * z);",
     lambda: pins.test_cov2d_closed_form_at_centre(0.3)),
    ("lowpass_dropped_on_x", "double a = C2[0][0] + lowpass, b = C2[0][1], c = C2[1][1] + lowpass;",
     "double a = C2[0][0], b = C2[0][1], c = C2[1][1] + lowpass;",
     lambda: pins.test_cov2d_closed_form_at_centre(0.0)),
    ("jacobian_unclamped", "double txz = fmin(limx, fmax(-limx, p[0] / z)) * z;", "double txz = p[0];",
     pins.test_jacobian_clamp_freezes_offaxis_term),
    ("depth_sum_order", "d32 = d32 + cam[9] * yf;\n        d32 = d32 + cam[10] * zf;",
     "d32 = d32 + cam[10] * zf;\n        d32 = d32 + cam[9] * yf;",
     pins.test_depth_bits_follow_the_fixed_float32_order),
    ("conic_offdiagonal_sign", "g[G_CONIC_B] = -b / det;", "g[G_CONIC_B] = b / det;",
     lambda: pins.test_single_gaussian_image_closed_form(0.7, 0.9)),
    ("pixel_centre_half_offset", "double px = fx * p[0] / z + cx,", "double px = fx * p[0] / z + cx + 0.5,",
     lambda: pins.test_single_gaussian_image_closed_form(0.0, 0.3)),
    ("adaptive_radius_factor_two_dropped", "double r_ad = sqrt(2.0 * lam * L);",
     "double r_ad = sqrt(lam * L);",
     lambda: pins.test_adaptive_radius_and_aabb_against_sampled_ellipse(0, A1)),
    ("aabb_axes_swapped", "double x_max = sqrt(2.0 * a * L);", "double x_max = sqrt(2.0 * c * L);",
     lambda: pins.test_adaptive_radius_and_aabb_against_sampled_ellipse(0, A1)),
    ("r_o_cap_dropped", "rx = ry = fmin(r_ad, r_o);", "rx = ry = r_ad;",
     pins.test_rcap_binds_for_opaque_gaussians),
    ("tile_interval_rounds_down", "double a = ceil(c - r), b = floor(c + r);",
     "double a = floor(c - r), b = floor(c + r);",
     lambda: pins.test_pair_tiles_equal_pixel_brute_force(3)),
    ("tile_key_transposed", "keys[off] = ((uint64_t)(ty * tiles_x + tx) << 32)",
     "keys[off] = ((uint64_t)(tx * tiles_x + ty) << 32)",
     lambda: pins.test_pair_tiles_equal_pixel_brute_force(3)),
    ("sort_ties_reversed", "if (x->v != y->v) return x->v < y->v ? -1 : 1;",
     "if (x->v != y->v) return x->v > y->v ? -1 : 1;",
     pins.test_sort_ties_keep_index_order),
    ("sh_cos_for_sin", "if (m > 0) return sqrt(2.0) * K * P * cos(m * phi);",
     "if (m > 0) return sqrt(2.0) * K * P * sin(m * phi);",
     pins.test_real_sh_matches_scipy),
    ("sh_sqrt2_dropped", "if (m < 0) return sqrt(2.0) * K * P * sin(am * phi);",
     "if (m < 0) return K * P * sin(am * phi);",
     pins.test_real_sh_orthonormal_by_quadrature),
    ("opacity_clamp_dropped", "double alpha = fmin(0.99, a_raw);", "double alpha = a_raw;",
     pins.test_early_termination_worked_example),
    ("alpha_low_skip_dropped", "if (alpha < alpha_low) return;", "if (alpha < 0.0) return;",
     lambda: pins.test_single_gaussian_image_closed_form(0.0, 0.3)),
    ("skipped_pairs_counted", "if (alpha < alpha_low) return;",
     "if (alpha < alpha_low) { s->load += 1; return; }",
     lambda: pins.test_single_gaussian_image_closed_form(-1.2, 0.05)),
    ("stop_after_blending", "if (test_T < t_min) { s->done = 1; return; }",
     "if (test_T < t_min) { s->done = 1; }",
     pins.test_early_termination_worked_example),
    ("blend_weight_without_transmittance", "s->C[c] += rgb[c] * alpha * s->T;",
     "s->C[c] += rgb[c] * alpha;",
     pins.test_two_gaussian_stack_worked_example),
    ("near_plane_at_zero", "if (!(d32 > near_z)) continue;", "if (!(d32 > 0.0f)) continue;",
     pins.test_near_plane_cull_and_depth_bits),
    ("eigenvalue_without_offdiagonal", "sqrt(0.25 * (a - c) * (a - c) + b * b);",
     "sqrt(0.25 * (a - c) * (a - c));",
     lambda: pins.test_adaptive_radius_and_aabb_against_sampled_ellipse(1, A1)),
    ("rect_3dgs_high_edge_not_rounded_up", "b = floor((c + R + (ORC_TILE - 1)) / ORC_TILE);",
     "b = floor((c + R) / ORC_TILE);",
     lambda: pins.test_3dgs_rect_rule_equals_point_set_brute_force(3)),
    ("tile_range_end_off_by_one", "ranges[2 * tile + 1] = (uint32_t)(i + 1);",
     "ranges[2 * tile + 1] = (uint32_t)i;",
     pins.test_sort_and_ranges_against_numpy),
    ("load_std_sample_form", "return sqrt(var / (double)hw);", "return sqrt(var / (double)(hw - 1));",
     pins.test_load_std_population_form),
]


@pytest.mark.parametrize("site,replacement,pin", [m[1:] for m in MUTANTS], ids=[m[0] for m in MUTANTS])
def test_a_pin_catches_the_planted_mistake(site, replacement, pin, tmp_path, monkeypatch):
    pin()                                            # passes on the real oracle
    src = open(SRC).read()
    assert src.count(site) == 1, f"mutation site not found once in adr_oracle.c: {site!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(site, replacement))
    lib = oracle.load_library(oracle.compile_library(str(path), str(tmp_path / "libmutant.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    with pytest.raises(AssertionError):
        pin()


# The image-loss oracle: a mutated copy of oracle/ssim.py is loaded and put in
# place of the module the SSIM pins use.
SSIM_MUTANTS = [
    ("c1_not_squared", "C1 = 0.01 ** 2", "C1 = 0.01",
     lambda: ssim_pins.test_constant_images_interior_closed_form(0.2, 0.7)),
    ("c2_not_squared", "C2 = 0.03 ** 2", "C2 = 0.03",
     lambda: ssim_pins.test_checkerboard_against_constant_closed_form(0.5, 0.3, 0.2)),
    ("window_sigma", "SIGMA = 1.5", "SIGMA = 1.0", ssim_pins.test_window_sum_matches_scipy_gaussian_filter),
    ("window_radius", "RADIUS = 5", "RADIUS = 4", ssim_pins.test_window_sum_matches_scipy_gaussian_filter),
    ("edge_padding", "    p = np.zeros((h + 2 * RADIUS, wd + 2 * RADIUS))\n"
                     "    p[RADIUS:RADIUS + h, RADIUS:RADIUS + wd] = a\n",
     "    p = np.pad(a, RADIUS, mode=\"edge\")\n", ssim_pins.test_window_sum_per_pixel_double_loop),
    ("covariance_without_means", "exy - mx * my", "exy",
     lambda: ssim_pins.test_checkerboard_against_constant_closed_form(0.5, 0.3, 0.2)),
    ("gradient_dxy_factor", "d_xy = 2 * s / a2", "d_xy = s / a2",
     lambda: ssim_pins.test_gradient_matches_central_differences(0.0, 1.0)),
    ("gradient_dxx_sign", "d_xx = -s / b2", "d_xx = s / b2",
     lambda: ssim_pins.test_gradient_matches_central_differences(0.0, 1.0)),
    ("gradient_second_moment_factor", "window_sum(d_mu) + 2 * x[c] * window_sum(d_xx)",
     "window_sum(d_mu) + x[c] * window_sum(d_xx)",
     lambda: ssim_pins.test_gradient_matches_central_differences(0.44, 0.11)),
    ("l1_gradient_not_averaged", "grad += w_l1 / n * np.sign(x - y)", "grad += w_l1 * np.sign(x - y)",
     ssim_pins.test_l1_subgradient_zero_at_ties),
]


@pytest.mark.parametrize("site,replacement,pin", [m[1:] for m in SSIM_MUTANTS],
                         ids=[m[0] for m in SSIM_MUTANTS])
def test_a_pin_catches_the_planted_image_loss_mistake(site, replacement, pin, tmp_path, monkeypatch):
    pin()                                            # passes on the real oracle
    src = open(ossim.__file__).read()
    assert site in src, f"mutation site not found in ssim.py: {site!r}"
    path = tmp_path / "ssim_mutant.py"
    path.write_text(src.replace(site, replacement))
    spec = importlib.util.spec_from_file_location("ssim_mutant", path)
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    monkeypatch.setattr(ssim_pins, "O", mutant)
    with pytest.raises(AssertionError):
        pin()


# The gradient oracle: a mutated copy of oracle/grad.py, loaded inside the
# oracle package (it imports the C oracle's wrappers relatively), is put in
# place of the module the gradient pins use.
GRAD_MUTANTS = [
    ("blend_weight_without_transmittance", "C = C + rgb[g][:, None] * (alpha * T * bw)[None]",
     "C = C + rgb[g][:, None] * (alpha * bw)[None]",
     lambda: grad_pins.test_torch_forward_equals_c_oracle(S.MODE_AABB)),
    ("conic_cross_term_factor", "q = conic[g, 0] * dx * dx + 2 * conic[g, 1] * dx * dy",
     "q = conic[g, 0] * dx * dx + conic[g, 1] * dx * dy",
     lambda: grad_pins.test_torch_forward_equals_c_oracle(S.MODE_PLAIN)),
    ("straight_through_sign", "L = L + bw * (1.0 + (alpha - a_det))", "L = L + bw * (1.0 - (alpha - a_det))",
     grad_pins.test_load_term_straight_through_definition),
    ("early_stop_sign", "cnt - cnt / theta * (S - S.detach())", "cnt + cnt / theta * (S - S.detach())",
     grad_pins.test_load_term_early_stop_reading_follows_the_slope_of_the_count),
    ("early_stop_without_optical_depth", "cnt - cnt / theta * (S - S.detach())",
     "cnt - cnt * (S - S.detach())",
     grad_pins.test_load_term_early_stop_reading_follows_the_slope_of_the_count),
    ("optical_depth_as_alpha", "S = S + bw * -torch.log1p(-alpha)", "S = S + bw * alpha",
     grad_pins.test_load_term_early_stop_reading_on_a_stack),
]


@pytest.mark.parametrize("site,replacement,pin", [m[1:] for m in GRAD_MUTANTS],
                         ids=[m[0] for m in GRAD_MUTANTS])
def test_a_pin_catches_the_planted_gradient_mistake(site, replacement, pin, tmp_path, monkeypatch):
    pin()                                            # passes on the real oracle
    src = open(ograd.__file__).read()
    assert src.count(site) == 1, f"mutation site not found once in grad.py: {site!r}"
    path = tmp_path / "grad_mutant.py"
    path.write_text(src.replace(site, replacement))
    spec = importlib.util.spec_from_file_location("oracle.grad_mutant", path)
    mutant = importlib.util.module_from_spec(spec)
    mutant.__package__ = "oracle"
    spec.loader.exec_module(mutant)
    monkeypatch.setattr(grad_pins, "og", mutant)
    with pytest.raises(AssertionError):
        pin()
