"""GPU parity at the parameter limits the library accepts, and at the degenerate
windows: 64-bit codes (7x9 plus the sentinel), 256 candidates per pass (the far and
the close range alike, and 128 disparities x 2 vertical offsets), grids of 8 x 8
blocks of 16 x 16 points, 32 occluders per box, decimation 8, 15-pixel windows, and
1x1 windows (codes hold the sentinel only, or nothing: every cost is 0 and the first
candidate wins).  Several frames per batch, boxes across the borders, stream and
graph launches; flags, block records and every forward and backward cost bit-exact,
disparity within 1e-4 px and depth within 1e-5."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs, compare_debug_arrays, oracle_evals

pytestmark = pytest.mark.gpu

BASE = dict(sentinel=1, far_side_px=50, close_factor=1, dy_min=0, dy_max=0, grid_g=8, pts_side=16,
            min_pts=4, fb_tol=1, agg_tau_d=1.0, agg_nmin=3, agg_mode=0, trim_frac=0.2,
            max_occluders=32, frontal_crop=0.0)

LIMITS = {
    "64-bit codes, 256 candidates, 8x8 grid": dict(
        win_w=7, win_h=9, far_dmin=-20, far_dmax=235, close_dmin=0, close_dmax=255),
    "128 disparities x 2 offsets, 15x3 window, k = 2": dict(
        win_w=15, win_h=3, far_dmin=0, far_dmax=127, close_dmin=-5, close_dmax=122, dy_min=-1,
        dy_max=0, close_factor=2, agg_mode=1, frontal_crop=0.5),
    "decimation 8, 3x15 window, no sentinel": dict(
        win_w=3, win_h=15, sentinel=0, far_dmin=0, far_dmax=63, close_dmin=0, close_dmax=31,
        close_factor=8, min_pts=1, agg_nmin=1),
    "1x1 window with sentinel": dict(
        win_w=1, win_h=1, far_dmin=0, far_dmax=40, close_dmin=2, close_dmax=70, grid_g=3, min_pts=1),
    "1x1 window without sentinel, one point per block": dict(
        win_w=1, win_h=1, sentinel=0, far_dmin=-3, far_dmax=12, close_dmin=0, close_dmax=31, pts_side=1,
        min_pts=1, agg_nmin=1),
}


@pytest.mark.parametrize("name", list(LIMITS))
def test_parameter_limits(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    params = dict(BASE)
    params.update(LIMITS[name])
    seed = sorted(LIMITS).index(name)
    W, H = 400, 300
    w = wl.multi_frame("frame1080", 9100 + seed, 2, W, H, 14, (6.0, 260.0), (0.5, 30.0), (2.0, 60.0),
                       strip_frac=0.3)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**params), debug=True)
    ctx = B.Context(params, len(w.frames), W, H, len(w.boxes))
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    for graph in (False, True):
        got = ctx.match_batch(batch, use_graph=graph, debug=True)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in got.items() if k != "debug"}
        where = f"{name} graph {graph}"
        compare_box_outputs(out, ref, where)
        dbg = got["debug"]
        compare_debug_arrays(dbg.blocks_np(), dbg.cost_f.cpu().numpy(), dbg.cost_b.cpu().numpy(), ref,
                             B.n_candidates(ctx.params), where)
        st = ctx.stats()
        assert st["error"] == 0, where
        assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params), where
    if params["win_w"] == 1:
        # a 1x1 window has no neighbours: a code is the sentinel or nothing.  Without
        # the sentinel every cost is 0 and the first candidate of the pass wins; with
        # it a point costs 1 exactly where the compared position lies off the plane.
        blk = ref["blocks"]
        searched = (blk["flags"] & orc.BLK_PRESENT) != 0
        searched &= (blk["flags"] & orc.BLK_FEW_POINTS) == 0
        assert searched.any()
        if params["sentinel"] == 0:
            assert np.all(ref["cost_f"] == 0) and np.all(ref["cost_b"] == 0)
            far = (ref["flags"] & orc.BOX_FAR) != 0
            dmin = np.where(far, params["far_dmin"], params["close_dmin"])[:, None]
            assert np.all((blk["d_f"] == dmin)[searched]) and np.all((blk["d_b"] == dmin)[searched])
            assert np.all(blk["dy_f"][searched] == params["dy_min"])
        else:
            assert ref["cost_f"].max() <= blk["n_valid"].max()
    ctx.close()


def _parity_batch(torch, w, params, where):
    from paper_2604_07980_gb300 import binding as B
    H = max(f.left.shape[0] for f in w.frames)
    W = max(f.left.shape[1] for f in w.frames)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**params), debug=True)
    ctx = B.Context(params, len(w.frames), W, H, len(w.boxes))
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    got = ctx.match_batch(batch, use_graph=True, debug=True)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in got.items() if k != "debug"}
    compare_box_outputs(out, ref, where)
    dbg = got["debug"]
    compare_debug_arrays(dbg.blocks_np(), dbg.cost_f.cpu().numpy(), dbg.cost_b.cpu().numpy(), ref,
                         B.n_candidates(ctx.params), where)
    st = ctx.stats()
    assert st["error"] == 0, where
    assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params), where
    ctx.close()
    return ref


@pytest.mark.parametrize("W,H", [(32768, 40), (80, 32768)])
def test_widest_and_tallest_frames(W, H):
    """The largest frame sides the library accepts (32768 px): the census tile list
    packs the tile index and the row into 10 and 16 bits; boxes at the far end of the
    long side and across it."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    params = dict(wl.PARAMS["frame1080"])
    params.update(far_dmax=31, close_dmax=63)
    w = wl.multi_frame("frame1080", 9200 + W % 7, 1, W, H, 24, (6.0, 38.0), (0.5, 20.0), (2.0, 40.0))
    extra = np.array([[W - 30, H - 36, W + 10, H - 2, 0], [W - 37, H - 39, W - 1, H - 1, 0],
                      [-5, -5, 30, 30, 0]], np.int32)
    w.boxes = np.concatenate([w.boxes, extra])
    ref = _parity_batch(torch, w, params, f"{W}x{H}")
    assert np.any(ref["flags"] & orc.BOX_VALID)


def test_many_small_frames_in_one_batch():
    """300 frames of 96x64 in one batch (frame indices well past a byte), two boxes each."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    params = dict(wl.PARAMS["frame1080"])
    params.update(far_dmax=15, close_dmax=31, grid_g=2)
    w = wl.multi_frame("frame1080", 9300, 300, 96, 64, 2, (8.0, 60.0), (0.5, 10.0), (2.0, 20.0))
    ref = _parity_batch(torch, w, params, "300 frames")
    assert np.any(ref["flags"] & orc.BOX_VALID)
