"""Planted mistakes in the oracle: every one must make a pin fail.

The oracle's pins (the other ``tests/test_oracle_*.py`` files) are chosen so
that a plausible mistake anywhere in ``oracle/oracle.c`` fails at least one of
them.  This file checks that claim mechanically.  Each entry below copies
oracle.c, replaces one exact snippet with a mistaken one (a flipped
comparison, a dropped penalty term, the other tie-break, an off-by-one in a
range, a swapped operand, a wrong constant), compiles the copy with the
oracle's own gcc flags, and runs the pin files in a child process whose
oracle module loads the copy.  The pins must fail for every mistake and pass
for the unchanged copy.  The committed oracle and its library are not
touched.

Every planted mistake changes some result the method defines (none is an
equivalent rewrite), and every one stays inside its buffers, so a copy fails
by a wrong value, never by a crash.  Left out on purpose: two changes found
to be equivalent rewrites: invalid pixels entering the median as -1 instead of 0
(both sort below every valid disparity) and a rectification fraction of
256/256 not carrying into the next tap (full weight on that tap gives the
same value).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = {k: f"tests/test_oracle_{k}.py"
        for k in ("census_cost", "sgm", "select", "e2e", "variants", "noise", "rectify", "render")}

# (name, pin file expected to catch it, exact snippet of oracle.c, mistake)
MUTANTS = [
    # census (Sec. VI-D): comparison, bit order, window order, border
    ("census_ties_set_the_bit", "census_cost",
     "bit = img[ny * W + nx] < centre ? 1 : 0;", "bit = img[ny * W + nx] <= centre ? 1 : 0;"),
    ("census_comparison_reversed", "census_cost",
     "bit = img[ny * W + nx] < centre ? 1 : 0;", "bit = img[ny * W + nx] > centre ? 1 : 0;"),
    ("census_column_major_window", "census_cost",
     "            for (int dy = -ry; dy <= ry; dy++) {\n"
     "                for (int dx = -rx; dx <= rx; dx++) {\n"
     "                    if (dx == 0 && dy == 0) continue;",
     "            for (int dx = -rx; dx <= rx; dx++) {\n"
     "                for (int dy = -ry; dy <= ry; dy++) {\n"
     "                    if (dx == 0 && dy == 0) continue;"),
    ("census_first_offset_least_significant", "census_cost",
     "used position */\n                    code = (code << 1) | (uint64_t)bit;",
     "used position */\n                    code = (code >> 1) | ((uint64_t)bit << (ww * wh - 2));"),
    ("census_outside_neighbour_sets_the_bit", "census_cost",
     "int bit = 0;\n                    if (nx >= 0", "int bit = 1;\n                    if (nx >= 0"),
    ("census_border_clamped", "census_cost",
     "if (nx >= 0 && nx < W && ny >= 0 && ny < H)\n"
     "                        bit = img[ny * W + nx] < centre ? 1 : 0;",
     "bit = img[(ny < 0 ? 0 : ny >= H ? H - 1 : ny) * W + (nx < 0 ? 0 : nx >= W ? W - 1 : nx)]"
     " < centre ? 1 : 0;"),
    # matching cost
    ("cost_outside_is_zero", "census_cost", "int c = nbits;", "int c = 0;"),
    ("cost_views_swapped", "census_cost",
     "hamming64(cL[y * W + x], cR[y * W + (x - d)])", "hamming64(cL[y * W + (x - d)], cR[y * W + x])"),
    ("cost_popcount_of_32_bits", "census_cost",
     "for (int k = 0; k < 64; k++) n +=", "for (int k = 0; k < 32; k++) n +="),
    # SGM recurrence
    ("sgm_no_right_neighbour", "sgm",
     "                if (d + 1 < D && lp[d + 1] + P1 < best) best = lp[d + 1] + P1;\n", ""),
    ("sgm_no_P2_term", "sgm", "                if (mprev + P2 < best) best = mprev + P2;\n", ""),
    ("sgm_P1_for_large_jumps", "sgm",
     "if (mprev + P2 < best) best = mprev + P2;", "if (mprev + P1 < best) best = mprev + P1;"),
    ("sgm_P1_missing_in_assignment", "sgm",
     "if (d - 1 >= 0 && lp[d - 1] + P1 < best) best = lp[d - 1] + P1;",
     "if (d - 1 >= 0 && lp[d - 1] + P1 < best) best = lp[d - 1];"),
    ("sgm_no_normalisation", "sgm", "l[d] = (int32_t)c[d] + best - mprev;", "l[d] = (int32_t)c[d] + best;"),
    ("sgm_path_starts_at_zero", "sgm",
     "for (int d = 0; d < D; d++) l[d] = c[d];\n                continue;",
     "for (int d = 0; d < D; d++) l[d] = 0;\n                continue;"),
    ("sgm_minimum_skips_d0", "sgm",
     "int32_t mprev = lp[0];\n            for (int k = 1; k < D; k++)",
     "int32_t mprev = lp[D - 1];\n            for (int k = 1; k < D - 1; k++)"),
    ("paths_four_path_set_wrong", "sgm",
     "{1, 0}, {-1, 0}, {0, 1}, {0, -1},", "{1, 0}, {-1, 0}, {0, 1}, {1, 1},"),
    ("paths_diagonal_repeated", "sgm",
     "{1, 1}, {-1, 1}, {1, -1}, {-1, -1},", "{1, 1}, {-1, 1}, {1, -1}, {1, 1},"),
    ("aggregate_skips_a_path", "sgm",
     "for (int r = 0; r < paths; r++) {", "for (int r = 1; r < paths; r++) {"),
    # winner-take-all, uniqueness, left-right check
    ("wta_largest_d_on_ties", "select", "if (s[d] < s[best]) best = d;", "if (s[d] <= s[best]) best = d;"),
    ("uniqueness_counts_the_neighbours", "select", "if (diff <= 1) continue;", "if (diff < 1) continue;"),
    ("uniqueness_other_ratio_form", "select",
     "(int64_t)(100 - uniq) * s[d] < (int64_t)100 * s[ds]",
     "(int64_t)100 * s[d] < (int64_t)(100 + uniq) * s[ds]"),
    ("uniqueness_equality_fails", "select",
     "(int64_t)(100 - uniq) * s[d] < (int64_t)100 * s[ds]",
     "(int64_t)(100 - uniq) * s[d] <= (int64_t)100 * s[ds]"),
    ("lr_equality_fails", "select", "if (diff > lr_max_diff) m |= 2;", "if (diff >= lr_max_diff) m |= 2;"),
    ("lr_search_range_one_short", "select",
     "if (W - 1 - xr < dmax) dmax = W - 1 - xr;", "if (W - 2 - xr < dmax) dmax = W - 2 - xr;"),
    ("lr_right_view_from_one_column", "select",
     "int32_t v = S[((size_t)y * W + (xr + d)) * D + d];", "int32_t v = S[((size_t)y * W + xr) * D + d];"),
    ("lr_right_view_largest_d_on_ties", "select",
     "if (v < sbest) { sbest = v; dr = d; }", "if (v <= sbest) { sbest = v; dr = d; }"),
    ("lr_outside_right_image_passes", "select",
     "if (xr < 0) {\n                    m |= 2;", "if (xr < 0) {\n                    m |= 0;"),
    # sub-pixel and depth
    ("subpixel_sign_flipped", "select",
     "df = (double)ds + (sm - sp) / (2.0 * (sm + sp - 2.0 * s0));",
     "df = (double)ds + (sp - sm) / (2.0 * (sm + sp - 2.0 * s0));"),
    ("subpixel_factor_two_dropped", "select",
     "df = (double)ds + (sm - sp) / (2.0 * (sm + sp - 2.0 * s0));",
     "df = (double)ds + (sm - sp) / (sm + sp - 2.0 * s0);"),
    ("subpixel_skips_d_one", "select", "ds >= 1 && ds <= D - 2", "ds >= 2 && ds <= D - 2"),
    ("subpixel_skips_d_max_minus_one", "select", "ds >= 1 && ds <= D - 2", "ds >= 1 && ds <= D - 3"),
    ("uniqueness_off_at_one_percent", "select", "if (uniq > 0) {", "if (uniq > 1) {"),
    ("zero_disparity_is_valid", "select", "            if (!(df > 0.0)) m |= 4;\n", ""),
    ("depth_from_integer_disparity", "select",
     "depth[y * W + x] = m == 0 ? fb / df : 0.0;", "depth[y * W + x] = m == 0 ? fb / (double)ds : 0.0;"),
    # variants: centre-symmetric census, block cost, median
    ("csct_comparison_reversed", "variants",
     "bit = img[ay * W + ax] < img[by * W + bx] ? 1 : 0;", "bit = img[ay * W + ax] > img[by * W + bx] ? 1 : 0;"),
    ("csct_centre_pair_included", "variants",
     "if (dy > 0 || (dy == 0 && dx >= 0)) continue;", "if (dy > 0 || (dy == 0 && dx > 0)) continue;"),
    ("csct_offsets_after_the_centre", "variants",
     "if (dy > 0 || (dy == 0 && dx >= 0)) continue;", "if (dy < 0 || (dy == 0 && dx <= 0)) continue;"),
    ("block_mean_truncated", "variants", "(uint8_t)((sum + n / 2) / n)", "(uint8_t)(sum / n)"),
    ("block_counts_outside_pixels", "variants",
     "if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;\n                        sum +=",
     "if (xx < 0 || xx >= W || yy < 0 || yy >= H) { n++; continue; }\n                        sum +="),
    ("median_one_above_the_middle", "variants", "out[y * W + x] = win[n / 2];", "out[y * W + x] = win[n / 2 + 1];"),
    ("median_border_reflected", "variants", "if (xx < 0) xx = 0;", "if (xx < 0) xx = -xx;"),
    # the whole stage: how the variants are wired together
    ("stage_csct_cost_with_full_census_width", "variants",
     "int nbits = census_cs ? (ww * wh - 1) / 2 : ww * wh - 1;", "int nbits = ww * wh - 1;"),
    ("stage_block_cost_only_when_both_sides_exceed_one", "variants",
     "if (rc == ORACLE_OK && (bw > 1 || bh > 1)) {", "if (rc == ORACLE_OK && (bw > 1 && bh > 1)) {"),
    ("stage_median_of_integer_disparities", "variants",
     "d0[i] = msk[i] == 0 ? dsp[i] : 0.0;", "d0[i] = msk[i] == 0 ? (double)ds[i] : 0.0;"),
    ("stage_median_keeps_unfiltered_depth", "variants",
     "depth[i] = dsp[i] > 0.0 ? f * baseline / dsp[i] : 0.0;", "depth[i] = depth[i];"),
    # sensor noise
    ("philox_wrong_weyl_constant", "noise", "k0 += W0;", "k0 += W1;"),
    ("philox_seven_rounds", "noise", "round < 10; round++", "round < 7; round++"),
    ("gamma_scale_missing_d", "noise", "gamma = d * v * theta;", "gamma = v * theta;"),
    ("noise_rounds_down", "noise", "double q = nearbyint(val);", "double q = floor(val);"),
    # rectification and registration
    ("tangential_coefficients_swapped", "rectify",
     "double xd = x * radial + 2.0 * c->p1 * x * y + c->p2 * (r2 + 2.0 * x * x);",
     "double xd = x * radial + 2.0 * c->p2 * x * y + c->p1 * (r2 + 2.0 * x * x);"),
    ("radial_k3_on_r4", "rectify", "c->k3 * r2 * r2 * r2", "c->k3 * r2 * r2"),
    ("rotation_not_transposed", "rectify",
     "double X = c->R[0] * xr + c->R[3] * yr + c->R[6];\n"
     "    double Y = c->R[1] * xr + c->R[4] * yr + c->R[7];\n"
     "    double Z = c->R[2] * xr + c->R[5] * yr + c->R[8];",
     "double X = c->R[0] * xr + c->R[1] * yr + c->R[2];\n"
     "    double Y = c->R[3] * xr + c->R[4] * yr + c->R[5];\n"
     "    double Z = c->R[6] * xr + c->R[7] * yr + c->R[8];"),
    ("bilinear_weights_transposed", "rectify",
     "(uint32_t)ax * by * t[1] + bx * (uint32_t)ay * t[2]",
     "bx * (uint32_t)ay * t[1] + (uint32_t)ax * by * t[2]"),
    ("bilinear_truncated", "rectify", "+ 32768u) >> 16", ") >> 16"),
    ("raw_focal_lengths_swapped", "rectify",
     "double ur = c->fx * xd + c->cx, vr = c->fy * yd + c->cy;",
     "double ur = c->fy * xd + c->cx, vr = c->fx * yd + c->cy;"),
    ("rgb_focal_lengths_swapped", "rectify",
     "double u2 = fx2 * (X2 / Z2) + cx2, v2 = fy2 * (Y2 / Z2) + cy2;",
     "double u2 = fy2 * (X2 / Z2) + cx2, v2 = fx2 * (Y2 / Z2) + cy2;"),
    ("registration_splats_points_behind_the_camera", "rectify",
     "            if (!(Z2 > 0.0)) continue;\n", "            if (Z2 == 0.0) continue;\n"),
    ("zbuffer_keeps_the_farthest", "rectify",
     "if (out[k] == 0.0f || z < out[k]) out[k] = z;", "if (out[k] == 0.0f || z > out[k]) out[k] = z;"),
    ("registration_splat_rounds_down", "rectify",
     "double pu = floor(u2 + 0.5), pv = floor(v2 + 0.5);", "double pu = floor(u2), pv = floor(v2);"),
    ("registration_translation_sign", "rectify", "R[2] * Z + t[0];", "R[2] * Z - t[0];"),
    # IR rendering
    ("lambert_without_pi", "render", "double fd = q->albedo / PI;", "double fd = q->albedo;"),
    ("irradiance_over_distance", "render",
     "double E = rp->power * pat * ni / dist2;", "double E = rp->power * pat * ni / dist;"),
    ("shadow_from_beyond_the_projector", "render",
     "if (t > 0.0 && t < 1.0) lit = 0;", "if (t > 0.0) lit = 0;"),
    ("ggx_denominator_without_n_dot_o", "render",
     "fs = D * F * (g1i * g1o) / (4.0 * ni * no);", "fs = D * F * (g1i * g1o) / (4.0 * ni);"),
    ("right_camera_on_the_left", "render",
     "double o[3] = {view ? rp->baseline : 0.0, 0.0, 0.0};", "double o[3] = {view ? -rp->baseline : 0.0, 0.0, 0.0};"),
    ("farthest_hit_wins", "render",
     "if (t > 0.0 && (best < 0 || t < tb))", "if (t > 0.0 && (best < 0 || t > tb))"),
    ("rectangle_twice_as_wide", "render",
     "if (s < -1.0 || s > 1.0 || w < -1.0 || w > 1.0) return -1.0;",
     "if (s < -2.0 || s > 2.0 || w < -1.0 || w > 1.0) return -1.0;"),
    ("no_ambient_term", "render", "double L = rp->ambient * q->albedo;", "double L = 0.0;"),
    ("schlick_exponent_4", "render", "double F = F0 + (1.0 - F0) * (m2 * m2 * m1);",
     "double F = F0 + (1.0 - F0) * (m2 * m2);"),
    ("schlick_exponent_6", "render", "double F = F0 + (1.0 - F0) * (m2 * m2 * m1);",
     "double F = F0 + (1.0 - F0) * (m2 * m2 * m2);"),
    ("dielectric_f0_0_05", "render", "double F0 = 0.04 * (1.0 - q->metallic)",
     "double F0 = 0.05 * (1.0 - q->metallic)"),
    ("fresnel_of_n_dot_h", "render", "double vh = dot3(ov, hv);", "double vh = nh;"),
]

# the child: point the oracle module at the copy, then run the pins on it
_CHILD = (
    "import sys, oracle, pytest\n"
    "oracle._SRC, oracle._LIB_PATH = sys.argv[1], sys.argv[2]\n"
    "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu', *sys.argv[3:]]))\n"
)


def _source():
    with open(os.path.join(ROOT, "oracle", "oracle.c")) as fh:
        return fh.read()


def _run_copy(tmp, name, text, first):
    """Compile ``text`` as the oracle and run the pins, ``first`` first;
    returns (pytest exit status, the end of its output)."""
    d = os.path.join(tmp, name)
    os.makedirs(d, exist_ok=True)
    src, lib = os.path.join(d, "oracle.c"), os.path.join(d, "_liboracle.so")
    with open(src, "w") as fh:
        fh.write(text)
    oracle.build(force=True, src=src, out=lib)
    files = [PINS[first]] + [f for k, f in PINS.items() if k != first]
    r = subprocess.run([sys.executable, "-c", _CHILD, src, lib, *files], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def test_every_snippet_occurs_exactly_once():
    src = _source()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, pin, old, new in MUTANTS:
        assert pin in PINS, name
        assert src.count(old) == 1, f"{name}: snippet found {src.count(old)} times"
        assert old != new, name


def test_pins_catch_every_planted_mistake(tmp_path):
    src = _source()
    jobs = [("unchanged", src, "census_cost")]
    jobs += [(name, src.replace(old, new), pin) for name, pin, old, new in MUTANTS]
    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda j: _run_copy(str(tmp_path), *j), jobs))
    rc0, out0 = results[0]
    assert rc0 == 0, f"the unchanged copy fails its pins:\n{out0}"
    # pytest exits with 1 when a test failed; any other status (a collection
    # error, a crash) would not show that a pin caught the mistake
    survivors = [(j[0], rc, out) for j, (rc, out) in zip(jobs[1:], results[1:]) if rc != 1]
    assert not survivors, "\n\n".join(f"{n}: exit {rc}\n{out}" for n, rc, out in survivors)
