"""Pins of the oracle's auto-rectification offset search (Sec. 5.1, census
matching in place of BM) and of its temporal filter."""
import numpy as np

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.brute import census_np


def _brute_counts(L, R, roi, dmin, dmax, deltas, d_thresh, fb_tol, ww, wh):
    H, W = L.shape
    CL, CR = census_np(L, ww, wh), census_np(R, ww, wh)

    def code(C, x, y):
        return int(C[y, x]) if 0 <= x < W and 0 <= y < H else 0

    out = []
    for delta in deltas:
        n = 0
        for y in range(roi[1], roi[3]):
            for x in range(roi[0], roi[2]):
                yl = y + delta
                if not (ww // 2 <= x < W - ww // 2 and wh // 2 <= yl < H - wh // 2):
                    continue
                cl = code(CL, x, yl)
                fwd = [bin(cl ^ code(CR, x - d, y)).count("1") for d in range(dmin, dmax + 1)]
                d_f = dmin + int(np.argmin(fwd))
                cq = code(CR, x - d_f, y)
                bwd = [bin(cq ^ code(CL, x - d_f + d, yl)).count("1") for d in range(dmin, dmax + 1)]
                d_b = dmin + int(np.argmin(bwd))
                n += abs(d_b - d_f) <= fb_tol and d_f > d_thresh
        out.append(n)
    return np.array(out)


def test_counts_equal_brute_force():
    rng = np.random.default_rng(21)
    L = np.clip(np.rint(wl.texture(rng, 30, 48)), 0, 255).astype(np.uint8)
    R = np.roll(L, (1, -3), axis=(0, 1))
    roi = (4, 2, 44, 27)
    best, counts = orc.auto_rect(L, R, roi, 0, 7, -2, 2, 1, fb_tol=1, win_w=5, win_h=3)
    ref = _brute_counts(L, R, roi, 0, 7, range(-2, 3), 1, 1, 5, 3)
    assert np.array_equal(counts, ref)
    assert best == -2 + int(np.argmax(ref))


def test_planted_vertical_offset_is_found():
    """R(x', y) = L(x' + d, y + delta_true): the left image shifted by delta_true matches."""
    rng = np.random.default_rng(22)
    H, W, d_true = 90, 160, 12
    for delta_true in (-3, 0, 2):
        big = np.clip(np.rint(wl.texture(rng, H + 10, W + 20)), 0, 255).astype(np.uint8)
        L = big[5:5 + H, 0:W]
        R = big[5 + delta_true:5 + delta_true + H, d_true:d_true + W]
        best, counts = orc.auto_rect(L, R, (30, 10, 140, 80), 0, 31, -4, 4, 4)
        assert best == delta_true, (delta_true, counts)
        # nearly every ROI pixel matches at the true offset; fewer one row off (the
        # texture is blurred, sigma 1.5), few three or more rows off
        peak = counts[delta_true + 4]
        assert peak > 0.9 * 110 * 70
        assert np.sort(counts)[-2] < 0.8 * peak
        far = [c for i, c in enumerate(counts) if abs(i - 4 - delta_true) >= 3]
        assert max(far) < 0.5 * peak


def test_filter_median_and_clamp():
    assert orc.rect_filter([3, 1, 2], 0, 5) == 2
    assert orc.rect_filter([3, 1, 2], 0, 1) == 1          # step clamped to +1
    assert orc.rect_filter([-6, -5, -7, 0], 0, 2) == -2   # even count: lower middle (-6), clamped
    assert orc.rect_filter([-6, -5, -7, 0], 0, 10) == -6  # even count: lower middle
    assert orc.rect_filter([2, 0], 0, 5) == 0
    assert orc.rect_filter([4], 3, 0) == 3                # no step allowed
    assert orc.rect_filter([], 7, 3) == 7


def test_equal_counts_take_the_first_offset():
    """delta* is the first offset with the largest count: on a pair whose rows are all
    equal every offset counts the same ROI pixels, and the lowest offset wins."""
    rng = np.random.default_rng(23)
    row = np.clip(np.rint(wl.texture(rng, 1, 120)[0]), 0, 255).astype(np.uint8)
    L = np.tile(row, (40, 1))
    R = np.roll(L, -3, axis=1)
    best, counts = orc.auto_rect(L, R, (20, 12, 100, 28), 0, 15, -2, 2, 1, win_w=5, win_h=3)
    assert np.all(counts == counts[0]) and counts[0] > 0
    assert best == -2
