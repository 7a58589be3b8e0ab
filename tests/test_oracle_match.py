"""Pins for the oracle's matching path: Eq. census_cost, argmin, Eq. subpixel,
forward-backward check (Sec. 4.3.3), occlusion-aware sampling (Sec. 4.3.5),
far/close split and aggregation (Sec. 4.3.4), Eq. 1."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.brute import census_np, cost_volume, longest_run_median


def _params(**kw):
    base = dict(wl.PARAMS["pair640"])
    base.update(kw)
    return orc.Params(**base)


def _textured_pair(W, H, d, seed=5, gain=1.0, offset=0.0):
    """Integer-shift pair: R(x) = L(x + d) (object at x in L is at x - d in R)."""
    rng = np.random.default_rng(seed)
    big = np.clip(np.rint(wl.texture(rng, H, W + d + 2)), 0, 255 - max(offset, 0))
    L = big[:, :W]
    R = np.clip(np.rint(gain * big[:, d:W + d] + offset), 0, 255)
    return L.astype(np.uint8), R.astype(np.uint8)


# ---------------------------------------------------------------- Eq. census_cost

def test_costs_equal_brute_force_volume():
    """Dense 3x3 blocks (every block pixel is a point): per-block cost vectors equal
    an independent numpy cost volume, including the vertical search."""
    W, H = 64, 40
    rng = np.random.default_rng(1)
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    p = _params(win_w=5, win_h=3, far_side_px=0, close_factor=1, close_dmin=-2, close_dmax=9,
                dy_min=-1, dy_max=1, grid_g=2, pts_side=16, min_pts=1, agg_nmin=1)
    box = np.array([[20, 8, 44, 30, 0]], np.int32)
    out = orc.match_frame(L, R, box, 2000.0, 0.3, p, debug=True)
    CL, CR = census_np(L, 5, 3), census_np(R, 5, 3)
    nd, ndy = 12, 3
    for s in range(4):
        a, b = s % 2, s // 2
        x0, x1 = 20 + a * 12, 20 + (a + 1) * 12
        y0, y1 = 8 + b * 11, 8 + (b + 1) * 11
        mask = np.zeros((H, W), bool)
        mask[y0:y1, x0:x1] = True
        mask[:1, :] = mask[-1:, :] = False
        mask[:, :2] = mask[:, -2:] = False
        vol = cost_volume(CL, CR, mask, -2, 9, -1, 1)
        got = out["cost_f"][0, s, :nd * ndy].reshape(ndy, nd)
        assert np.array_equal(got, vol), s
        assert out["blocks"][0, s]["n_valid"] == mask.sum()


def test_self_match_zero_cost_at_zero():
    rng = np.random.default_rng(2)
    L = np.clip(np.rint(wl.texture(rng, 60, 90)), 0, 255).astype(np.uint8)
    p = _params()
    box = np.array([[30, 6, 78, 54, 0]], np.int32)
    out = orc.match_frame(L, L, box, 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(out["cost_f"][0, :, 0] == 0)
    assert np.all(b["d_f"] == 0) and np.all(b["d_b"] == 0)
    assert np.all(b["flags"] & orc.BLK_VALID)


@pytest.mark.parametrize("d", [0, 7, 23, 40])
def test_planted_integer_shift_is_argmin(d):
    L, R = _textured_pair(160, 64, d, seed=d, gain=1.0, offset=10.0)
    p = _params()
    box = np.array([[90, 8, 138, 56, 0]], np.int32)
    out = orc.match_frame(L, R, box, 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(b["d_f"] == d) and np.all(b["d_b"] == d)
    assert np.all(out["cost_f"][0, :, d] == 0)  # offset without clipping changes nothing
    if d > 0:
        assert out["flags"][0] & orc.BOX_VALID
        assert out["disp"][0] == pytest.approx(d, abs=0.05)
    else:  # Eq. 1 needs d > 0
        assert out["flags"][0] & orc.BOX_NONPOS_DISP and not out["flags"][0] & orc.BOX_VALID


def test_argmin_is_round_of_fractional_truth_on_clean_texture():
    """Clean planted textures (no noise, gain 1, offset 0): argmin = round(d_true)."""
    w = wl.pair640(seed=1000)
    w2 = wl.pair640(seed=1000)  # same geometry
    # rebuild the same pair without noise
    rng = np.random.default_rng(1234)
    fr = w.frames[0]
    H, W = fr.left.shape
    Lf = wl.texture(rng, H, W)
    Rf = Lf.copy()
    boxes = w.boxes[:, :4].tolist()
    d = [float(v) for v in w.d_true]
    d = [np.floor(v) + (0.2 if (v % 1) < 0.5 else 0.8) for v in d]  # stay away from .5
    for i in sorted(range(len(boxes)), key=lambda i: boxes[i][3]):
        wl._paint(Lf, Rf, rng, boxes[i], d[i])
    L = np.clip(np.rint(Lf), 0, 255).astype(np.uint8)
    R = np.clip(np.rint(Rf), 0, 255).astype(np.uint8)
    out = orc.match_frame(L, R, w2.boxes, 2000.0, 0.3, orc.Params(**w.params), debug=True)
    for i, di in enumerate(d):
        assert np.all(out["blocks"][i]["d_f"] == int(np.rint(di))), (i, di)


# ---------------------------------------------------------------- Eq. subpixel

@pytest.mark.parametrize("sm,s0,sp", [(7, 3, 5), (25, 1, 9), (9, 1, 1), (4, 2, 4), (100, 0, 3)])
def test_parabola_vertex_closed_form(sm, s0, sp):
    """The vertex of the parabola through (-1,sm), (0,s0), (1,sp) is at
    (sm - sp) / (2 (sm - 2 s0 + sp)) (exact rational arithmetic)."""
    v = Fraction(sm - sp, 2 * (sm - 2 * s0 + sp))
    got = orc.subpixel(40, sm, s0, sp)
    assert got == pytest.approx(float(40 + v), abs=2e-6)


def test_parabola_exact_quadratic():
    """Costs sampled from 16 (d - 10.25)^2 + 1 give the vertex 10.25 exactly."""
    S = lambda d: int(16 * (d - 10.25) ** 2 + 1)
    assert orc.subpixel(10, S(9), S(10), S(11)) == 10.25


def test_block_subpixel_uses_neighbour_costs():
    L, R = _textured_pair(160, 64, 12, seed=9)
    out = orc.match_frame(L, R, np.array([[90, 8, 138, 56, 0]], np.int32), 2000.0, 0.3,
                          _params(), debug=True)
    for b, cf in zip(out["blocks"][0], out["cost_f"][0]):
        d = b["d_f"]
        assert (b["s_m"], b["s_0"], b["s_p"]) == (cf[d - 1], cf[d], cf[d + 1])
        assert b["d_sub"] == np.float32(orc.subpixel(d, cf[d - 1], cf[d], cf[d + 1]))


def test_range_edge_keeps_integer_argmin():
    L, R = _textured_pair(160, 64, 20, seed=4)
    p = _params(close_dmin=0, close_dmax=20)
    out = orc.match_frame(L, R, np.array([[90, 8, 138, 56, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(b["d_f"] == 20)
    assert np.all(b["d_sub"] == 20.0)
    assert np.all(b["flags"] & orc.BLK_SUBPIX_CLAMPED)


# ---------------------------------------------------------------- Sec. 4.3.3

def test_backward_cost_at_forward_match_equals_forward_cost():
    w = wl.frame1080(W=480, H=270, n_boxes=12, side_range=(12, 120))
    fr = w.frames[0]
    out = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m,
                          orc.Params(**w.params), debug=True)
    checked = 0
    for i in range(w.n_boxes):
        for s in range(out["blocks"].shape[1]):
            b = out["blocks"][i, s]
            if not (b["flags"] & orc.BLK_PRESENT) or b["flags"] & orc.BLK_FEW_POINTS:
                continue
            far = out["flags"][i] & orc.BOX_FAR
            nd = (w.params["far_dmax"] if far else w.params["close_dmax"]) + 1
            assert out["cost_b"][i, s, b["d_f"]] == out["cost_f"][i, s, b["d_f"]]
            assert b["d_f"] < nd
            checked += 1
    assert checked > 20


def test_backward_meets_forward_with_vertical_search():
    """S_b(d_f, dy_f) = S_f(d_f, dy_f) on unrelated noise images with a vertical
    search: the backward query sits at the matched right position (x - d_f,
    y + dy_f), so at the forward match it pairs the same codes."""
    rng = np.random.default_rng(41)
    L = rng.integers(0, 256, (48, 90), dtype=np.uint8)
    R = rng.integers(0, 256, (48, 90), dtype=np.uint8)
    p = _params(win_w=5, win_h=5, close_dmin=-3, close_dmax=12, dy_min=-2, dy_max=2, grid_g=3,
                pts_side=4, min_pts=1)
    out = orc.match_frame(L, R, np.array([[30, 6, 78, 42, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.any(b["dy_f"] != 0)
    for s in range(9):
        c = (int(b[s]["dy_f"]) + 2) * 16 + int(b[s]["d_f"]) + 3
        assert out["cost_b"][0, s, c] == out["cost_f"][0, s, c] == out["blocks"][0, s]["s_0"], s


def test_mirrored_pair_forward_equals_original_backward():
    """Swap and mirror the pair: the object keeps its disparity, and with dense
    points the mirrored forward costs are the original backward costs of the
    mirrored block (block column a <-> g-1-a)."""
    d = 9
    L, R = _textured_pair(200, 60, d, seed=21)
    Wd = 200
    p = _params(close_dmax=31)
    box = np.array([[100, 6, 148, 54, 0]], np.int32)
    out = orc.match_frame(L, R, box, 2000.0, 0.3, p, debug=True)
    assert np.all(out["blocks"][0]["d_f"] == d)
    Lm = np.ascontiguousarray(R[:, ::-1])
    Rm = np.ascontiguousarray(L[:, ::-1])
    x0r, x1r = 100 - d, 148 - d  # the object in R
    boxm = np.array([[Wd - x1r, 6, Wd - x0r, 54, 0]], np.int32)
    outm = orc.match_frame(Lm, Rm, boxm, 2000.0, 0.3, p, debug=True)
    for s in range(9):
        a, b = s % 3, s // 3
        sm = b * 3 + (2 - a)
        assert np.array_equal(outm["cost_f"][0, sm], out["cost_b"][0, s])
    assert np.all(outm["blocks"][0]["d_f"] == d)


@pytest.mark.parametrize("dy", [1, -2])
def test_vertical_offset_found_forward_and_backward(dy):
    """Sec. 4.3.3 with a vertical search: R(x - d, y + dy) = L(x, y).  The forward
    search finds (d, dy) at zero cost; the backward search, queried at the matched
    right position, finds the same (d, dy) at zero cost."""
    d = 5
    rng = np.random.default_rng(40 + dy)
    big = np.clip(np.rint(wl.texture(rng, 80, 200)), 0, 255).astype(np.uint8)
    L = big[10:70, 0:180]
    R = big[10 - dy:70 - dy, d:180 + d]  # R[y + dy, x - d] = L[y, x]
    p = _params(close_dmin=0, close_dmax=15, dy_min=-2, dy_max=2)
    out = orc.match_frame(L, R, np.array([[90, 6, 138, 54, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(b["d_f"] == d) and np.all(b["dy_f"] == dy)
    assert np.all(b["d_b"] == d) and np.all(b["dy_b"] == dy)
    c = (dy + 2) * 16 + d
    assert np.all(out["cost_f"][0, :, c] == 0) and np.all(out["cost_b"][0, :, c] == 0)


def test_fb_rejects_inconsistent_match():
    """An object whose right-image content is unrelated texture fails the check in
    at least some blocks; FB_REJECT is then set on the box."""
    rng = np.random.default_rng(8)
    L = np.clip(np.rint(wl.texture(rng, 60, 160)), 0, 255).astype(np.uint8)
    R = np.clip(np.rint(wl.texture(rng, 60, 160)), 0, 255).astype(np.uint8)
    out = orc.match_frame(L, R, np.array([[90, 6, 138, 54, 0]], np.int32), 2000.0, 0.3,
                          _params(fb_tol=0), debug=True)
    b = out["blocks"][0]
    rej = (b["flags"] & orc.BLK_FB_REJECT) != 0
    assert rej.any()
    assert np.all(np.abs(b["d_b"][rej] - b["d_f"][rej]) > 0)
    assert out["flags"][0] & orc.BOX_FB_REJECT


# ---------------------------------------------------------------- Sec. 4.3.5 / 4.3.4

def test_occluder_points_are_excluded():
    rng = np.random.default_rng(3)
    L = np.clip(np.rint(wl.texture(rng, 120, 200)), 0, 255).astype(np.uint8)
    a = [100, 20, 148, 68]
    occ = [120, 40, 135, 80]  # bottom 80 > 68: occludes a
    up = [90, 10, 110, 60]    # bottom 60 < 68: does not occlude a (a occludes it)
    boxes = np.array([a + [0], occ + [0], up + [0]], np.int32)
    out = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(), debug=True)
    for s in range(9):
        bx0, by0 = 100 + (s % 3) * 16, 20 + (s // 3) * 16
        xs, ys = np.meshgrid(np.arange(bx0, bx0 + 16), np.arange(by0, by0 + 16))
        hidden = (xs >= occ[0]) & (xs < occ[2]) & (ys >= occ[1]) & (ys < occ[3])
        assert out["blocks"][0, s]["n_valid"] == 256 - hidden.sum()
    # the upper box loses the part covered by a
    nv_up = out["blocks"][2]["n_valid"].sum()
    assert nv_up < out["blocks"][2]["n_pts"].sum()


def test_equal_bottoms_do_not_occlude_and_cap_keeps_nearest():
    rng = np.random.default_rng(4)
    L = np.clip(np.rint(wl.texture(rng, 120, 200)), 0, 255).astype(np.uint8)
    a = [100, 20, 148, 68]
    same = [90, 30, 120, 68]
    near1 = [140, 20, 160, 90]
    near2 = [100, 60, 110, 80]
    boxes = np.array([a + [0], same + [0], near1 + [0], near2 + [0]], np.int32)
    full = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(), debug=True)
    cap1 = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(max_occluders=1), debug=True)
    xs, ys = np.meshgrid(np.arange(100, 148), np.arange(20, 68))
    inside = lambda r: (xs >= r[0]) & (xs < r[2]) & (ys >= r[1]) & (ys < r[3])
    assert full["blocks"][0]["n_valid"].sum() == (~(inside(near1) | inside(near2))).sum()
    # cap 1 keeps near1 (bottom 90 > 80)
    assert cap1["blocks"][0]["n_valid"].sum() == (~inside(near1)).sum()


def test_frontal_crop_priority_when_occluders_exceed_the_cap():
    """Sec. 4.3.5 priority rule: with more occluders than slots, occluders whose box
    centre lies in the centred crop are kept first, the others fill the remaining slots
    nearest first; with frontal_crop = 0 the nearest are kept."""
    rng = np.random.default_rng(12)
    L = np.clip(np.rint(wl.texture(rng, 120, 200)), 0, 255).astype(np.uint8)
    a = [100, 20, 148, 68]
    f1 = [70, 30, 110, 80]     # centre (90, 55): inside the 0.2 crop [80, 120) x [48, 72); bottom 80
    f2 = [90, 50, 130, 75]     # centre (110, 62.5): inside; bottom 75
    n1 = [140, 10, 190, 110]   # centre (165, 60): outside; bottom 110
    n2 = [120, 60, 200, 100]   # centre (160, 80): outside; bottom 100
    boxes = np.array([b + [0] for b in (a, f1, f2, n1, n2)], np.int32)
    xs, ys = np.meshgrid(np.arange(100, 148), np.arange(20, 68))
    inside = lambda r: (xs >= r[0]) & (xs < r[2]) & (ys >= r[1]) & (ys < r[3])

    def usable(kept):
        m = np.zeros_like(xs, bool)
        for r in kept:
            m |= inside(r)
        return int((~m).sum())

    def n_valid(**kw):
        out = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(**kw), debug=True)
        return int(out["blocks"][0]["n_valid"].sum())

    assert n_valid(max_occluders=2) == usable([n1, n2])
    assert n_valid(max_occluders=2, frontal_crop=0.2) == usable([f1, f2])
    assert n_valid(max_occluders=3, frontal_crop=0.2) == usable([f1, f2, n1])
    assert n_valid(max_occluders=1, frontal_crop=0.2) == usable([f1])
    # a crop that holds every centre ranks by proximity alone again
    assert n_valid(max_occluders=2, frontal_crop=1.0) == usable([n1, n2])
    with pytest.raises(ValueError):
        n_valid(frontal_crop=1.5)


def test_far_close_threshold_and_empty_boxes():
    rng = np.random.default_rng(6)
    L = np.clip(np.rint(wl.texture(rng, 200, 300)), 0, 255).astype(np.uint8)
    p = orc.Params(**wl.PARAMS["frame1080"])
    boxes = np.array([[100, 50, 139, 80, 0],     # max side 39 -> FAR
                      [100, 100, 140, 120, 0],   # max side 40 -> CLOSE
                      [400, 10, 450, 40, 0],     # outside -> EMPTY
                      [-30, 150, 20, 190, 0],    # clipped to 20 x 40 -> CLOSE
                      [50, 60, 50, 90, 0]],      # zero width -> EMPTY
                     np.int32)
    out = orc.match_frame(L, L, boxes, 2000.0, 0.3, p, debug=True)
    f = out["flags"]
    assert f[0] & orc.BOX_FAR and not f[1] & orc.BOX_FAR
    assert f[2] & orc.BOX_EMPTY and f[4] & orc.BOX_EMPTY
    assert np.isnan(out["disp"][2])
    assert not f[3] & orc.BOX_FAR and not f[3] & orc.BOX_EMPTY


def test_dense_sampling_of_48px_box():
    """A 48x48 box on a 3x3 grid at full resolution gives 16x16 dense blocks."""
    rng = np.random.default_rng(1)
    L = np.clip(np.rint(wl.texture(rng, 100, 200)), 0, 255).astype(np.uint8)
    out = orc.match_frame(L, L, np.array([[80, 20, 128, 68, 0]], np.int32), 2000.0, 0.3,
                          _params(), debug=True)
    assert np.all(out["blocks"][0]["n_pts"] == 256)
    assert np.all(out["blocks"][0]["n_valid"] == 256)


@pytest.mark.parametrize("seed", range(8))
def test_aggregation_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 26))
    vals = np.round(rng.normal(30, 3, n) * 4) / 4
    vals = vals.astype(np.float32)
    for mode in (0, 1):
        got = orc.aggregate(vals, 1.0, 3, mode, 0.2)
        run = longest_run_median(vals, 1.0, 3)
        if run is None:
            assert got is None
            continue
        if mode == 0:
            assert got == pytest.approx(float(np.median(run)), abs=1e-6)
        else:
            from scipy.stats import trim_mean
            assert got == pytest.approx(float(trim_mean(run, 0.2)), abs=1e-5)


def test_aggregation_hand_lists():
    assert orc.aggregate([9.1, 5.2, 5.0, 9.0, 5.4], 1.0, 3) == pytest.approx(5.2)
    assert orc.aggregate([4.5, 1.0, 4.0, 1.5], 1.0, 2) == pytest.approx(1.25)  # tie -> lower run
    assert orc.aggregate([1.0, 3.0, 5.0], 1.0, 2) is None
    assert orc.aggregate([2.0, 2.5, 2.75, 3.0], 1.0, 4) == pytest.approx(2.625)
    assert orc.aggregate([], 1.0, 1) is None


def test_depth_eq1_paper_examples():
    """Sec. 1.2: b = 30 cm, f = 2000 px -> 200 m at d = 3.0 px; b = 12 cm -> d = 1.2 px."""
    assert orc.depth(2000.0, 0.30, 3.0) == pytest.approx(200.0, rel=1e-6)
    assert orc.depth(2000.0, 0.12, 1.2) == pytest.approx(200.0, rel=1e-6)
    assert np.isnan(orc.depth(2000.0, 0.3, 0.0)) and np.isnan(orc.depth(2000.0, 0.3, -1.0))


def test_pair640_end_to_end_accuracy_band():
    """Parity-unpinned sanity band: sub-pixel estimates near the planted truth."""
    w = wl.pair640()
    fr = w.frames[0]
    out = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m,
                          orc.Params(**w.params))
    assert np.all(out["flags"] & orc.BOX_VALID)
    assert np.median(np.abs(out["disp"] - w.d_true)) < 0.25
    np.testing.assert_allclose(out["depth"], fr.f_px * fr.baseline_m / out["disp"], rtol=1e-6)


def test_argmin_ties_take_first_candidate():
    """All-equal costs (a flat scene): the first candidate in (dy, d) order wins."""
    L = np.full((40, 120), 90, np.uint8)
    p = _params(close_dmin=3, close_dmax=20, dy_min=-1, dy_max=1, min_pts=1)
    out = orc.match_frame(L, L, np.array([[60, 8, 108, 32, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(b["d_f"] == 3) and np.all(b["dy_f"] == -1)
    assert np.all(b["d_b"] == 3) and np.all(b["dy_b"] == -1)


def test_fb_tolerance_is_inclusive():
    """|d_b - d_f| <= fb_tol is accepted: a block's flag flips exactly at fb_tol."""
    w = wl.frame1080(W=480, H=270, n_boxes=16, side_range=(12, 150))
    fr = w.frames[0]
    seen = 0
    for tol in (0, 1, 2):
        prm = dict(w.params)
        prm["fb_tol"] = tol
        out = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m,
                              orc.Params(**prm), debug=True)
        b = out["blocks"].reshape(-1)
        run = (b["flags"] & orc.BLK_PRESENT) != 0
        run &= (b["flags"] & orc.BLK_FEW_POINTS) == 0
        dxv = np.abs(b["d_b"] - b["d_f"])
        valid = (b["flags"] & orc.BLK_VALID) != 0
        assert np.array_equal(valid[run], dxv[run] <= tol)
        seen += int(np.sum(run & (dxv == tol) & valid))
    assert seen > 0


def test_half_resolution_rescale():
    """CLOSE matching at k = 2: an even shift d is found as d/2 on the decimated grid
    and reported back as d full-res px (d_full = k d_sub)."""
    L, R = _textured_pair(300, 100, 24, seed=13)
    p = _params(close_factor=2, far_side_px=0, close_dmax=31, grid_g=3, min_pts=4)
    out = orc.match_frame(L, R, np.array([[150, 10, 246, 90, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert np.all(b["d_f"] == 12)
    np.testing.assert_array_equal(b["d_full"], b["d_sub"] * np.float32(2))
    assert out["disp"][0] == pytest.approx(24.0, abs=0.2)


# ---------------------------------------------------------------- Sec. 4.3.4 point grid

@pytest.mark.parametrize("k,dx", [(1, 0), (2, 0), (2, 1)])
def test_point_grid_located_by_occluders(k, dx):
    """Sec. 4.3.4/4.3.5: a 32-px block (on the matching grid) with 16 points per side
    holds its points at the centres of 2-px cells, offsets 1, 3, ..., 31; an occluder
    hides a point when the point's full-resolution position k x lies in it.  A
    one-column occluder that reaches below the box therefore hides exactly the points
    of one column (16 per block, two blocks deep) or none; one reaching down from row
    r hides the point rows at or below r.  Which full-resolution columns and rows
    hold points is listed here in closed form, not from the sampling formula.
    With k = 2 and an odd left edge (dx = 1) the box starts on the matching grid at
    ceil(x0 / k): decimated pixel x is in the box iff its source pixel k x is."""
    side = 64 * k  # two 32-px blocks per axis on the matching grid
    x0, y0 = 40 * k - dx, 10 * k
    H, W = y0 + side + 40, x0 + side + 40
    rng = np.random.default_rng(21)
    L = np.clip(np.rint(wl.texture(rng, H, W)), 0, 255).astype(np.uint8)
    p = _params(far_side_px=0, close_factor=k, grid_g=2, pts_side=16, min_pts=1,
                close_dmax=15, max_occluders=4)
    box = [x0, y0, x0 + side, y0 + side, 0]
    cols = {k * (40 + 1 + 2 * q) for q in range(16)} | {k * (40 + 33 + 2 * q) for q in range(16)}
    for c in range(x0 - 1, x0 + side + 1):
        occ = [c, y0 - 5, c + 1, y0 + side + 5, 0]
        out = orc.match_frame(L, L, np.array([box, occ], np.int32), 2000.0, 0.3, p, debug=True)
        nv = out["blocks"][0]["n_valid"]
        hidden = 32 if c in cols else 0
        assert int(nv.sum()) == 4 * 256 - hidden, c
        assert np.all(out["blocks"][0]["n_pts"] == 256)
    # rows: an occluder covering every row from r down past the box hides the 32
    # points of each point row at or below r
    rows = {k * (10 + 1 + 2 * m) for m in range(16)} | {k * (10 + 33 + 2 * m) for m in range(16)}
    for r in range(y0 - 1, y0 + side + 1):
        occ = [x0 - 3, r, x0 + side + 3, y0 + side + 5, 0]
        out = orc.match_frame(L, L, np.array([box, occ], np.int32), 2000.0, 0.3, p, debug=True)
        hidden = 32 * sum(1 for y in rows if y >= r)
        assert int(out["blocks"][0]["n_valid"].sum()) == 4 * 256 - hidden, r


def test_min_points_boundary_and_box_flags():
    """Sec. 4.3.4: a block with fewer usable points than min_pts is not searched and
    flags FEW_POINTS; with every block so flagged the box has no consistent segment."""
    L, R = _textured_pair(160, 64, 7, seed=31, offset=10.0)
    box = np.array([[90, 8, 138, 56, 0]], np.int32)  # 48x48, 3x3 blocks of 16x16 points
    ok = orc.match_frame(L, R, box, 2000.0, 0.3, _params(min_pts=256), debug=True)
    b = ok["blocks"][0]
    assert np.all(b["n_valid"] == 256)
    assert not np.any(b["flags"] & orc.BLK_FEW_POINTS) and np.all(b["flags"] & orc.BLK_VALID)
    assert ok["flags"][0] & orc.BOX_VALID and not ok["flags"][0] & orc.BOX_FEW_POINTS
    few = orc.match_frame(L, R, box, 2000.0, 0.3, _params(min_pts=257), debug=True)
    b = few["blocks"][0]
    assert np.all(b["flags"] & orc.BLK_FEW_POINTS) and not np.any(b["flags"] & orc.BLK_VALID)
    assert np.all(few["cost_f"][0] == 0)  # never searched
    f = few["flags"][0]
    assert f & orc.BOX_FEW_POINTS and f & orc.BOX_NO_SEGMENT and not f & orc.BOX_VALID
    assert np.isnan(few["disp"][0]) and np.isnan(few["depth"][0])


def test_aggregation_needs_agg_nmin_consistent_blocks():
    """Sec. 4.3.4: the box takes the aggregate of its longest run of consistent blocks
    only when the run holds at least agg_nmin of them; nine agreeing blocks pass at
    agg_nmin = 9 and fail at 10."""
    L, R = _textured_pair(160, 64, 7, seed=32, offset=10.0)
    box = np.array([[90, 8, 138, 56, 0]], np.int32)
    nine = orc.match_frame(L, R, box, 2000.0, 0.3, _params(agg_nmin=9), debug=True)
    assert np.all(nine["blocks"][0]["d_f"] == 7)
    assert nine["flags"][0] & orc.BOX_VALID
    assert nine["disp"][0] == pytest.approx(float(np.median(nine["blocks"][0]["d_full"])), abs=1e-6)
    ten = orc.match_frame(L, R, box, 2000.0, 0.3, _params(agg_nmin=10), debug=True)
    assert ten["flags"][0] & orc.BOX_NO_SEGMENT and not ten["flags"][0] & orc.BOX_VALID
    assert np.isnan(ten["disp"][0])


def test_far_box_is_one_block_at_full_resolution():
    """Sec. 4.3.4: a box smaller than the far threshold is one block of up to
    pts_side x pts_side points on the full-resolution grid, searched over the far
    range; its disparity is that block's, with no aggregation."""
    L, R = _textured_pair(200, 60, 5, seed=33, offset=10.0)
    p = _params(far_side_px=40, close_factor=2, far_dmin=0, far_dmax=20, agg_nmin=9)
    box = np.array([[120, 12, 150, 42, 0]], np.int32)  # 30 x 30 < 40: FAR
    out = orc.match_frame(L, R, box, 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0]
    assert out["flags"][0] & orc.BOX_FAR and out["flags"][0] & orc.BOX_VALID
    assert b[0]["n_pts"] == 256 and b[0]["d_f"] == 5
    assert np.all(b[1:]["flags"] == 0)  # no further blocks
    assert out["disp"][0] == b[0]["d_full"] == b[0]["d_sub"]  # k = 1, no rescale


def test_touching_box_is_no_occluder_under_the_cap():
    """Sec. 4.3.5: occlusion needs overlapping boxes; a nearer box that only touches
    the target's edge (half-open rectangles) takes no occluder slot."""
    rng = np.random.default_rng(14)
    L = np.clip(np.rint(wl.texture(rng, 120, 200)), 0, 255).astype(np.uint8)
    a = [100, 20, 148, 68]
    touch = [148, 10, 170, 100]  # shares a's right edge only; bottom 100
    occ = [120, 40, 140, 80]     # overlaps; bottom 80
    boxes = np.array([a + [0], touch + [0], occ + [0]], np.int32)
    out = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(max_occluders=1), debug=True)
    xs, ys = np.meshgrid(np.arange(100, 148), np.arange(20, 68))
    hidden = (xs >= occ[0]) & (xs < occ[2]) & (ys >= occ[1]) & (ys < occ[3])
    assert int(out["blocks"][0]["n_valid"].sum()) == int((~hidden).sum())


def test_frontal_crop_upper_edge_is_open():
    """Sec. 4.3.5 priority rule, crop edges: a centre on the crop's right edge
    (doubled centre x0 + x1 = W (1 + c), exact in fp32 at c = 0.5) is not frontal, so
    with one slot the frontal occluder is kept although the edge one is nearer."""
    rng = np.random.default_rng(15)
    L = np.clip(np.rint(wl.texture(rng, 120, 200)), 0, 255).astype(np.uint8)
    a = [100, 20, 148, 68]
    edge = [140, 30, 160, 90]   # doubled centre (300, 120): x on the open edge; bottom 90
    front = [110, 40, 130, 75]  # doubled centre (240, 115): inside; bottom 75
    boxes = np.array([a + [0], edge + [0], front + [0]], np.int32)
    out = orc.match_frame(L, L, boxes, 2000.0, 0.3, _params(max_occluders=1, frontal_crop=0.5), debug=True)
    xs, ys = np.meshgrid(np.arange(100, 148), np.arange(20, 68))
    hidden = (xs >= front[0]) & (xs < front[2]) & (ys >= front[1]) & (ys < front[3])
    assert int(out["blocks"][0]["n_valid"].sum()) == int((~hidden).sum())


def test_far_box_searches_the_far_range():
    """Sec. 4.3.4: FAR blocks search [far_dmin, far_dmax]; a shift of 1 px below
    far_dmin = 2 is not found, the search ends at the range's lower end."""
    L, R = _textured_pair(200, 60, 1, seed=34, offset=10.0)
    p = _params(far_side_px=40, far_dmin=2, far_dmax=20, close_dmin=0, close_dmax=63)
    out = orc.match_frame(L, R, np.array([[120, 12, 150, 42, 0]], np.int32), 2000.0, 0.3, p, debug=True)
    b = out["blocks"][0][0]
    assert out["flags"][0] & orc.BOX_FAR
    assert b["d_f"] == 2 and b["flags"] & orc.BLK_SUBPIX_CLAMPED
