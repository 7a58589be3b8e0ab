"""GPU parity over seeded random parameter sets: every window shape the library
accepts (the fixed 5x5/7x7/9x7 tile code and the generic staged path), decimation
1-3, random and negative disparity ranges, vertical search, grid sizes, point
counts, minimum points, consistency tolerances, both aggregation modes, occluder
caps and the frontal crop, sentinel on and off; small random frames with boxes
across the borders, several frames per batch; the default tuning through the
stream and graph paths, then the two-pass matcher with the second census variant
and the narrowest strip (most column chunks).  Flags, block records and every
forward and backward cost bit-exact; disparity within 1e-4 px, depth 1e-5."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs, compare_debug_arrays, oracle_evals

pytestmark = pytest.mark.gpu

WINDOWS = [(5, 5), (7, 7), (9, 7), (3, 3), (5, 3), (3, 7), (11, 5), (7, 9)]


def _random_params(rng):
    win = WINDOWS[rng.integers(len(WINDOWS))]
    ndy_half = int(rng.integers(0, 3))
    dy_min, dy_max = (-ndy_half, ndy_half) if rng.random() < 0.5 else (0, ndy_half)
    ndy = dy_max - dy_min + 1
    max_nd = 256 // ndy

    def d_range():
        nd = int(rng.integers(1, min(max_nd, 96) + 1))
        dmin = int(rng.integers(-6, 8))
        return dmin, dmin + nd - 1

    far_dmin, far_dmax = d_range()
    close_dmin, close_dmax = d_range()
    g = int(rng.integers(1, 6))
    return dict(win_w=win[0], win_h=win[1], sentinel=int(rng.integers(0, 2)),
                far_side_px=int(rng.choice([0, 16, 30, 50])), close_factor=int(rng.integers(1, 4)),
                far_dmin=far_dmin, far_dmax=far_dmax, close_dmin=close_dmin, close_dmax=close_dmax,
                dy_min=dy_min, dy_max=dy_max, grid_g=g, pts_side=int(rng.integers(2, 17)),
                min_pts=int(rng.integers(1, 24)), fb_tol=int(rng.integers(0, 3)),
                agg_tau_d=float(rng.choice([0.5, 1.0, 2.0])), agg_nmin=int(rng.integers(1, g * g + 1)),
                agg_mode=int(rng.integers(0, 2)), trim_frac=float(rng.choice([0.0, 0.1, 0.25])),
                max_occluders=int(rng.integers(0, 33)),
                frontal_crop=float(rng.choice([0.0, 0.0, 0.4])))


@pytest.mark.parametrize("seed", range(40))
def test_random_configuration(seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(7000 + seed)
    params = _random_params(rng)
    n_frames = int(rng.integers(1, 4))
    W, H = int(rng.integers(60, 260)), int(rng.integers(50, 200))
    w = wl.multi_frame("frame1080", 8000 + seed, n_frames, W, H, int(rng.integers(3, 25)), (4.0, 120.0),
                       (0.5, 12.0), (1.0, 24.0), strip_frac=0.3)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**params), debug=True)
    ctx = B.Context(params, n_frames, W, H, max(len(w.boxes), 1))
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    nd_max = max(params["far_dmax"] - params["far_dmin"], params["close_dmax"] - params["close_dmin"]) + 1
    narrow = ((nd_max + 2 + 7) // 8) * 8
    runs = [dict(census_mode=2), dict(census_mode=0),
            dict(match_mode=1, census_mode=1, strip_cols=narrow, match_threads=256)]
    for i, tuning in enumerate(runs):
        graph = i == 1
        if tuning:
            ctx.set_tuning(**tuning)
        got = ctx.match_batch(batch, use_graph=graph, debug=True)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in got.items() if k != "debug"}
        where = f"seed {seed} graph {graph} tuning {tuning} params {params}"
        compare_box_outputs(out, ref, where)
        dbg = got["debug"]
        compare_debug_arrays(dbg.blocks_np(), dbg.cost_f.cpu().numpy(), dbg.cost_b.cpu().numpy(), ref,
                             B.n_candidates(ctx.params), where)
        st = ctx.stats()
        assert st["error"] == 0, where
        assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params), where
    ctx.close()


@pytest.mark.parametrize("seed", range(24))
def test_random_configuration_mapped(seed):
    """The mapped host entry point over random parameter sets (every window shape,
    decimation 1-3, vertical search, ...): the gather must copy every source byte
    the census of the marked tiles reads, whatever the window's reach and the
    decimation.  The staging images hold noise from a copying call first."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(9100 + seed)
    params = _random_params(rng)
    n_frames = int(rng.integers(1, 4))
    W, H = 16 * int(rng.integers(4, 17)), int(rng.integers(50, 200))
    w = wl.multi_frame("frame1080", 9300 + seed, n_frames, W, H, int(rng.integers(3, 25)), (4.0, 120.0),
                       (0.5, 12.0), (1.0, 24.0), strip_frac=0.3)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**params))
    ctx = B.Context(params, n_frames, W, H, max(len(w.boxes), 1))
    packed = np.stack([np.stack([f.left, f.right]) for f in w.frames])
    pinned = torch.empty(packed.shape, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[...] = packed
    noise = torch.empty(packed.shape, dtype=torch.uint8, pin_memory=True)
    noise.numpy()[...] = rng.integers(0, 256, packed.shape, dtype=np.uint8)
    fpx = [f.f_px for f in w.frames]
    bm = [f.baseline_m for f in w.frames]
    ctx.match_batch_host_packed(noise.numpy(), w.boxes, fpx, bm)
    got = ctx.match_batch_host_packed(pinned.numpy(), w.boxes, fpx, bm, mapped=True)
    where = f"seed {seed} mapped params {params}"
    compare_box_outputs(got, ref, where)
    st = ctx.stats()
    assert st["error"] == 0, where
    assert st["host_bytes"] <= packed.nbytes, where
    ctx.close()
