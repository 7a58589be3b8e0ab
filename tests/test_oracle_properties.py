"""Randomised pins of the oracle (CPU): properties the method fixes, checked on
many small generated inputs rather than a few fixed ones.

- Census (Sec. 4.3.1): equal to the numpy brute force for random windows,
  decimations and sizes; unchanged by an added offset without clipping and by any
  strictly increasing remap of intensities; a defined pixel's comparison bits
  count only neighbours strictly above the centre.
- Matching (Eq. census_cost, Sec. 4.3.3): per-block forward costs equal an
  independent numpy cost volume; the backward cost at the forward match equals the
  forward cost there; costs never exceed points x code bits.
"""
import numpy as np
import pytest

try:
    from hypothesis import given, settings, strategies as st
except ImportError:  # hypothesis is optional: without it these tests skip one by one when run
    # (not at collection, so a run that deselects them reports no skip)
    class _AnyStrategy:
        def __getattr__(self, name):
            return lambda *a, **k: None

    st = _AnyStrategy()

    def settings(*a, **k):
        return lambda f: f

    def given(*a, **k):
        def deco(f):
            def skipped():
                pytest.skip("hypothesis is not installed")
            skipped.__name__, skipped.__doc__ = f.__name__, f.__doc__
            return skipped
        return deco

from oracle import oracle as orc  # noqa: E402
from paper_2604_07980_gb300 import workloads as wl  # noqa: E402
from tests.brute import census_np, cost_volume  # noqa: E402

WINDOWS = [(3, 3), (5, 5), (7, 7), (9, 7), (3, 5), (5, 3)]


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), h=st.integers(1, 24), w=st.integers(1, 30),
       win=st.sampled_from(WINDOWS), k=st.integers(1, 3), sentinel=st.integers(0, 1))
def test_census_equals_brute_force(seed, h, w, win, k, sentinel):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
    if h > 4 and w > 4:
        img[1:4, 1:4] = img[2, 2]  # ties
    got = orc.census(img, k, *win, sentinel)
    ref = census_np(np.ascontiguousarray(img[::k, ::k]), *win, sentinel)
    assert np.array_equal(got, ref)


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), win=st.sampled_from(WINDOWS), offset=st.integers(0, 155),
       steps=st.lists(st.integers(1, 2), min_size=99, max_size=99))
def test_census_order_invariance(seed, win, offset, steps):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 100, size=(20, 27), dtype=np.uint8)
    base = orc.census(img, 1, *win, 1)
    assert np.array_equal(base, orc.census((img + offset).astype(np.uint8), 1, *win, 1))
    lut = np.cumsum([0] + steps).astype(np.int64)  # strictly increasing on 0..99, at most 198
    assert np.array_equal(base, orc.census(lut.astype(np.uint8)[img], 1, *win, 1))


@settings(max_examples=30, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), win=st.sampled_from(WINDOWS))
def test_census_bits_count_greater_neighbours(seed, win):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 8, size=(15, 17), dtype=np.uint8)  # many ties
    c = orc.census(img, 1, *win, 1)
    ww, wh = win
    sx, sy = ww // 2, wh // 2
    n = ww * wh
    for y in range(sy, 15 - sy):
        for x in range(sx, 17 - sx):
            code = int(c[y, x])
            assert code >> n == 1  # the sentinel, alone above the comparison bits
            greater = int(np.sum(img[y - sy:y + sy + 1, x - sx:x + sx + 1] > img[y, x]))
            assert bin(code & ((1 << n) - 1)).count("1") == greater


@settings(max_examples=15, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), dmin=st.integers(-3, 2), nd=st.integers(1, 12),
       dy=st.integers(0, 1), win=st.sampled_from([(3, 3), (5, 3), (5, 5)]))
def test_forward_costs_equal_volume_and_backward_meets_forward(seed, dmin, nd, dy, win):
    rng = np.random.default_rng(seed)
    H, W = 36, 60
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    dmax = dmin + nd - 1
    params = dict(wl.PARAMS["pair640"])
    params.update(win_w=win[0], win_h=win[1], far_side_px=0, close_factor=1, close_dmin=dmin,
                  close_dmax=dmax, dy_min=-dy, dy_max=dy, grid_g=1, pts_side=16, min_pts=1, agg_nmin=1)
    p = orc.Params(**params)
    box = np.array([[18, 6, 40, 28, 0]], np.int32)  # 22 x 22: a 16 x 16 point grid
    out = orc.match_frame(L, R, box, 2000.0, 0.3, p, debug=True)
    blk = out["blocks"][0, 0]
    ndy = 2 * dy + 1
    costs = out["cost_f"][0, 0, :nd * ndy].reshape(ndy, nd)
    # the points of the grid whose left census is defined
    sx, sy = win[0] // 2, win[1] // 2
    xs = [18 + (2 * j + 1) * 22 // 32 for j in range(16)]
    ys = [6 + (2 * m + 1) * 22 // 32 for m in range(16)]
    mask = np.zeros((H, W), bool)
    for y in ys:
        for x in xs:
            if sx <= x < W - sx and sy <= y < H - sy:
                mask[y, x] = True
    CL, CR = census_np(L, *win), census_np(R, *win)
    vol = cost_volume(CL, CR, mask, dmin, dmax, -dy, dy)
    assert np.array_equal(costs, vol)
    assert blk["n_valid"] == mask.sum()
    assert costs.max() <= mask.sum() * (win[0] * win[1] + 1)
    # S_b(d_f) = S_f(d_f): the backward pass sees the same pairs at the forward match
    cb = out["cost_b"][0, 0, :nd * ndy].reshape(ndy, nd)
    d_f, dy_f = int(blk["d_f"]), int(blk["dy_f"])
    assert cb[dy_f + dy, d_f - dmin] == costs[dy_f + dy, d_f - dmin]
    # the forward match is the first minimum in (dy, d) order
    flat = costs.reshape(-1)
    assert (dy_f + dy) * nd + (d_f - dmin) == int(np.argmin(flat))
