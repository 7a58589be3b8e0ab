"""The oracle's pins, checked against planted mistakes (CPU).

Each case below plants one plausible mistake in a copy of the oracle's C source (a
flipped comparison, a dropped term, a wrong sign or index, transposed operands),
compiles the copy with the oracle's own flags, loads it in place of the oracle and
runs the pin named beside it, which must then fail.  The oracle's source is never
modified; the copies are built under oracle/_build/mut/.  Every case also checks that
its mistake applies to exactly one place in the source, so an edit of the oracle that
moves the text makes the case fail rather than pass silently.
"""
import importlib
import os
import re

import pytest

from oracle import oracle as orc

M = "tests.test_oracle_match"
C = "tests.test_oracle_census"
P = "tests.test_oracle_points"
R = "tests.test_oracle_rect"

# (name, text in ctm_oracle.c, replacement, pin module, pin function, pin arguments)
MUTATIONS = [
    # census, Sec. 4.3.1
    ("xi not strict", "return a > b ? 1 : 0;", "return a >= b ? 1 : 0;",
     C, "test_fig2_worked_example", {}),
    ("xi operands transposed", "(uint64_t)xi(v, centre);", "(uint64_t)xi(centre, v);",
     C, "test_fig2_worked_example", {}),
    ("census centre not decimated", "int centre = img[(size_t)(k * y) * pitch + (size_t)(k * x)];",
     "int centre = img[(size_t)(y) * pitch + (size_t)(x)];",
     C, "test_scaled_census_is_census_of_decimated_image", {"k": 2, "shape": (24, 30)}),
    ("sentinel dropped", "c = sentinel ? 1u : 0u;", "c = 0u;", C, "test_fig2_worked_example", {}),
    ("census border off by one", "x + sx >= Ws || y - sy < 0", "x + sx > Ws || y - sy < 0",
     C, "test_fig2_worked_example", {}),
    # Eq. subpixel, Eq. 1, aggregation (Sec. 4.3.4)
    ("parabola offset sign", "return (float)d_star - off;", "return (float)d_star + off;",
     M, "test_parabola_vertex_closed_form", {"sm": 7, "s0": 3, "sp": 5}),
    ("parabola curvature term", "(s_p + s_m - 2 * s_0)", "(s_p + s_m - s_0)",
     M, "test_parabola_vertex_closed_form", {"sm": 7, "s0": 3, "sp": 5}),
    ("depth drops the baseline", "return fb / d;", "return f_px / d;", M, "test_depth_eq1_paper_examples", {}),
    ("run gap inclusive", "if (v[i] - v[i - 1] < tau_d) {", "if (v[i] - v[i - 1] <= tau_d) {",
     M, "test_aggregation_brute_force", {"seed": 1}),
    ("run tie takes the last", "if (cur_len > best_len) {", "if (cur_len >= best_len) {",
     M, "test_aggregation_brute_force", {"seed": 5}),
    ("even median takes the upper", "else r = (run[m / 2 - 1] + run[m / 2]) * 0.5f;", "else r = run[m / 2];",
     M, "test_aggregation_brute_force", {"seed": 1}),
    ("trim rounds up", "int t = (int)floorf(trim_frac * (float)m);", "int t = (int)ceilf(trim_frac * (float)m);",
     M, "test_aggregation_brute_force", {"seed": 0}),
    ("trimmed mean divides by all", "r = s / (float)cnt;", "r = s / (float)m;",
     M, "test_aggregation_brute_force", {"seed": 0}),
    # boxes, occlusion (Sec. 4.3.5), point grid (Sec. 4.3.4)
    ("touching boxes overlap", "return ix1 > ix0 && iy1 > iy0;", "return ix1 >= ix0 && iy1 >= iy0;",
     M, "test_touching_box_is_no_occluder_under_the_cap", {}),
    ("occluder closed on the right", "x >= r.x0 && x < r.x1", "x >= r.x0 && x <= r.x1",
     M, "test_occluder_points_are_excluded", {}),
    ("box floored on the matching grid", "int sx0 = ceil_div(r.x0, k), sx1 = ceil_div(r.x1, k);",
     "int sx0 = r.x0 / k, sx1 = r.x1 / k;", M, "test_point_grid_located_by_occluders", {"k": 2, "dx": 1}),
    ("occlusion tested on the matching grid", "inside(cb[occ[t]], k * x, k * y)", "inside(cb[occ[t]], x, y)",
     M, "test_point_grid_located_by_occluders", {"k": 2, "dx": 0}),
    ("frontal crop closed on the right", "sx < (float)W * (1.0f + c)", "sx <= (float)W * (1.0f + c)",
     M, "test_frontal_crop_upper_edge_is_open", {}),
    ("frontal occluders ranked last", "if (fa != fb) return fa > fb;", "if (fa != fb) return fa < fb;",
     M, "test_frontal_crop_priority_when_occluders_exceed_the_cap", {}),
    ("farthest occluders kept", "if (cb[a].y1 != cb[b].y1) return cb[a].y1 > cb[b].y1;",
     "if (cb[a].y1 != cb[b].y1) return cb[a].y1 < cb[b].y1;",
     M, "test_equal_bottoms_do_not_occlude_and_cap_keeps_nearest", {}),
    ("equal bottoms occlude", "if (rects_overlap(r, cb[j]) && cb[j].y1 > r.y1) occ[nocc++] = j;",
     "if (rects_overlap(r, cb[j]) && cb[j].y1 >= r.y1) occ[nocc++] = j;",
     M, "test_equal_bottoms_do_not_occlude_and_cap_keeps_nearest", {}),
    ("occluder cap dropped", "if (nocc > p->max_occluders) nocc = p->max_occluders;", "",
     M, "test_equal_bottoms_do_not_occlude_and_cap_keeps_nearest", {}),
    ("boxes not clipped", "r.x1 = b[2] > W ? W : b[2];", "r.x1 = b[2];",
     M, "test_far_close_threshold_and_empty_boxes", {}),
    ("far threshold inclusive", "is_far[i] = side < p->far_side_px;", "is_far[i] = side <= p->far_side_px;",
     M, "test_far_close_threshold_and_empty_boxes", {}),
    ("blocks in column-major order", "int a = s % g, bb = s / g;", "int a = s / g, bb = s % g;",
     M, "test_costs_equal_brute_force_volume", {}),
    ("point rows at cell edges", "int y = by0 + ((2 * m + 1) * (by1 - by0)) / (2 * ny);",
     "int y = by0 + ((2 * m) * (by1 - by0)) / (2 * ny);", M, "test_point_grid_located_by_occluders", {"k": 1, "dx": 0}),
    ("point columns at cell edges", "int x = bx0 + ((2 * q + 1) * (bx1 - bx0)) / (2 * nx);",
     "int x = bx0 + ((2 * q) * (bx1 - bx0)) / (2 * nx);", M, "test_point_grid_located_by_occluders", {"k": 1, "dx": 0}),
    ("min_pts inclusive", "if (np < p->min_pts) {", "if (np <= p->min_pts) {",
     M, "test_min_points_boundary_and_box_flags", {}),
    # Eq. census_cost and the searches (Sec. 4.3.3)
    ("forward disparity sign", "code_at(CR, Ws, Hs, px[t] - d, py[t] + dy));",
     "code_at(CR, Ws, Hs, px[t] + d, py[t] + dy));", M, "test_costs_equal_brute_force_volume", {}),
    ("forward vertical sign", "code_at(CR, Ws, Hs, px[t] - d, py[t] + dy));",
     "code_at(CR, Ws, Hs, px[t] - d, py[t] - dy));", M, "test_costs_equal_brute_force_volume", {}),
    ("forward drops the left code", "s += popc64(code_at(CL, Ws, Hs, px[t], py[t]) ^\n",
     "s += popc64(0 ^\n", M, "test_costs_equal_brute_force_volume", {}),
    ("backward disparity sign", "code_at(CL, Ws, Hs, qx + d, qy - dy));", "code_at(CL, Ws, Hs, qx - d, qy - dy));",
     M, "test_planted_integer_shift_is_argmin", {"d": 7}),
    ("backward vertical sign", "code_at(CL, Ws, Hs, qx + d, qy - dy));", "code_at(CL, Ws, Hs, qx + d, qy + dy));",
     M, "test_backward_meets_forward_with_vertical_search", {}),
    ("backward query off the matched row", "int qx = px[t] - d_f, qy = py[t] + dy_f;",
     "int qx = px[t] - d_f, qy = py[t];", M, "test_backward_meets_forward_with_vertical_search", {}),
    ("forward argmin takes the last tie", "if (best < 0 || Sf[c] < Sf[best]) best = c;",
     "if (best < 0 || Sf[c] <= Sf[best]) best = c;", M, "test_argmin_ties_take_first_candidate", {}),
    ("backward argmin takes the last tie", "if (bestb < 0 || Sb[c] < Sb[bestb]) bestb = c;",
     "if (bestb < 0 || Sb[c] <= Sb[bestb]) bestb = c;", M, "test_argmin_ties_take_first_candidate", {}),
    ("left neighbour cost from the right", "o->s_m = d_f > dmin ? Sf[best - 1] : 0;",
     "o->s_m = d_f > dmin ? Sf[best + 1] : 0;", M, "test_block_subpixel_uses_neighbour_costs", {}),
    ("upper range end not clamped", "if (d_f == dmin || d_f == dmax) {", "if (d_f == dmin || d_f == dmax + 1) {",
     M, "test_range_edge_keeps_integer_argmin", {}),
    ("consistency tolerance exclusive", "if (dxv <= p->fb_tol) {", "if (dxv < p->fb_tol) {",
     M, "test_fb_tolerance_is_inclusive", {}),
    ("no rescale to full resolution", "o->d_full = o->d_sub * (float)k;", "o->d_full = o->d_sub;",
     M, "test_half_resolution_rescale", {}),
    ("far boxes split into blocks", "const int g = far ? 1 : p->grid_g;", "const int g = p->grid_g;",
     M, "test_far_box_is_one_block_at_full_resolution", {}),
    ("far boxes search the close range", "const int dmin = far ? p->far_dmin : p->close_dmin;",
     "const int dmin = p->close_dmin;", M, "test_far_box_searches_the_far_range", {}),
    ("zero disparity accepted", "if (d_box > 0.0f) {", "if (d_box >= 0.0f) {",
     M, "test_planted_integer_shift_is_argmin", {"d": 0}),
    # Sec. 4.3.6 reprojection and covariance
    ("box centre half a pixel off", "(x0 + x1 - 1) / 2.0, (y0 + y1 - 1) / 2.0", "(x0 + x1) / 2.0, (y0 + y1 - 1) / 2.0",
     P, "test_standard_q_closed_form_and_eq1", {}),
    ("Q transposed", "h[r] += g->Q[4 * r + c] * in[c];", "h[r] += g->Q[4 * c + r] * in[c];",
     P, "test_standard_q_closed_form_and_eq1", {}),
    ("translation dropped", " + g->T[4 * r + 2] * p[2] + g->T[4 * r + 3];", " + g->T[4 * r + 2] * p[2];",
     P, "test_vehicle_transform", {}),
    ("reprojected box not clipped", "const int x1 = b[2] < g->width ? b[2] : g->width,",
     "const int x1 = b[2],", P, "test_invalid_cases_are_nan_and_boxes_are_clipped", {}),
    ("variance with Z squared", "o[6] = Z * Z * Z * Z * g->disp_var / (fb * fb);",
     "o[6] = Z * Z * g->disp_var / (fb * fb);", P, "test_variance_is_squared_depth_derivative", {}),
    # Sec. 5.1 offset search and filter
    ("offset threshold inclusive", "if (dx <= fb_tol && d_f > d_thresh) ++count;",
     "if (dx <= fb_tol && d_f >= d_thresh) ++count;", R, "test_counts_equal_brute_force", {}),
    ("offset backward search unshifted", "code_at(CL, W, H, x - d_f + d, y + delta));",
     "code_at(CL, W, H, x - d_f + d, y));", R, "test_counts_equal_brute_force", {}),
    ("offset forward argmin takes the last tie", "if (s_d < s_best) { s_best = s_d; d_f = d; }",
     "if (s_d <= s_best) { s_best = s_d; d_f = d; }", R, "test_counts_equal_brute_force", {}),
    ("offset tie takes the last", "if (count > best_count) {", "if (count >= best_count) {",
     R, "test_equal_counts_take_the_first_offset", {}),
    ("filter takes the upper middle", "const int med = v[(n - 1) / 2];", "const int med = v[n / 2];",
     R, "test_filter_median_and_clamp", {}),
    ("filter step not clamped", "if (step > max_step) step = max_step;", "",
     R, "test_filter_median_and_clamp", {}),
]


def _slug(name: str) -> str:
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")


def test_every_pin_passes_on_the_oracle_itself():
    """The named pins pass on the unmodified oracle (so a failure below is the mistake's)."""
    for _, _, _, mod, fn, kw in MUTATIONS:
        getattr(importlib.import_module(mod), fn)(**kw)


@pytest.mark.parametrize("name,old,new,mod,fn,kw", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(name, old, new, mod, fn, kw, monkeypatch):
    src = open(orc._SRC).read()
    assert src.count(old) == 1, f"{name}: the text to mutate is not unique in the oracle"
    out_dir = os.path.join(orc._BUILD, "mut")
    os.makedirs(out_dir, exist_ok=True)
    c_path = os.path.join(out_dir, _slug(name) + ".c")
    with open(c_path, "w") as f:
        f.write(src.replace(old, new))
    so = orc.compile_source(c_path, os.path.join(out_dir, _slug(name) + ".so"))
    monkeypatch.setattr(orc, "_SO", so)
    monkeypatch.setattr(orc, "_lib", None)
    monkeypatch.setattr(orc, "build", lambda force=False: so)
    pin = getattr(importlib.import_module(mod), fn)
    with pytest.raises(AssertionError):
        pin(**kw)
