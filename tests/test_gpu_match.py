"""GPU parity of the matching path (Algorithm 2) against the oracle.

Integer outputs (flags, argmins, point counts, every forward and backward cost)
must be bit-exact; sub-pixel disparity within 1e-4 px and depth within 1e-5
relative.  Cases cover several tiles and ragged tails, boxes at and beyond the
image border, empty and degenerate boxes, vertical search, trimmed mean, and
the plain per-box path, the single-frame path and the batched graph path.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs, compare_debug, oracle_evals, torch_frames

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _run_frame(torch, w, fi=0, debug=True, params=None, plain=False, ctx=None):
    from paper_2604_07980_gb300 import binding as B
    params = params or w.params
    fr = w.frames[fi]
    sel = w.boxes[:, 4] == fi
    boxes = np.ascontiguousarray(w.boxes[sel])
    H, W = fr.left.shape
    own = ctx is None
    if own:
        ctx = B.Context(params, 1, W, H, max(len(boxes), 1))
    L, R = torch_frames([fr])[0]
    bt = torch.from_numpy(boxes).cuda()
    if plain:
        got = ctx.match_boxes_plain(L, R, bt, fr.f_px, fr.baseline_m)
    else:
        got = ctx.match_boxes(L, R, bt, fr.f_px, fr.baseline_m, debug=debug)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items() if k != "debug"}
    out["debug"] = got.get("debug")
    stats = ctx.stats()
    ref = orc.match_frame(fr.left, fr.right, boxes, fr.f_px, fr.baseline_m, orc.Params(**params),
                          debug=debug)
    if own:
        ctx.close()
    return out, ref, stats, B.n_candidates(ctx.params)


def test_pair640_bit_exact(torch_cuda):
    w = wl.pair640()
    got, ref, stats, nc = _run_frame(torch_cuda, w)
    compare_box_outputs(got, ref, "pair640")
    compare_debug(got["debug"], ref, nc, "pair640")
    assert stats["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params)
    assert np.all(got["flags"] & orc.BOX_VALID)


def test_frame1080_bit_exact(torch_cuda):
    w = wl.frame1080()
    got, ref, stats, nc = _run_frame(torch_cuda, w)
    compare_box_outputs(got, ref, "frame1080")
    compare_debug(got["debug"], ref, nc, "frame1080")
    assert stats["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params)
    assert stats["n_boxes"] == w.n_boxes


def test_plain_path_equals_oracle(torch_cuda):
    w = wl.frame1080(W=960, H=540, n_boxes=24, side_range=(12, 200))
    got, ref, _, _ = _run_frame(torch_cuda, w, debug=False, plain=True)
    compare_box_outputs(got, ref, "plain")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_small_cases_with_edges(torch_cuda, seed):
    """Odd sizes, boxes touching/crossing borders, empty and tiny boxes, ranges
    reaching past the left border, occluders."""
    rng = np.random.default_rng(100 + seed)
    W, H = 203 + 17 * seed, 119 + 5 * seed
    w = wl.multi_frame("frame1080", 2000 + seed, 1, W, H, 20, (6.0, 90.0), (0.5, 20.0), (2.0, 60.0),
                       strip_frac=0.3)
    extra = np.array([[-10, -5, 30, 40, 0], [W - 20, H - 10, W + 15, H + 9, 0], [50, 50, 50, 80, 0],
                      [W + 5, 10, W + 40, 30, 0], [10, 10, 13, 12, 0], [0, 0, W, H, 0],
                      [5, 20, 44, 59, 0]], np.int32)
    w.boxes = np.concatenate([w.boxes, extra])
    params = dict(w.params, far_side_px=24, close_dmax=47, far_dmax=25, max_occluders=4,
                  min_pts=int(rng.integers(4, 20)))
    got, ref, stats, nc = _run_frame(torch_cuda, w, params=params)
    compare_box_outputs(got, ref, f"edges{seed}")
    compare_debug(got["debug"], ref, nc, f"edges{seed}")
    assert stats["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params)


def test_vertical_search_and_negative_range(torch_cuda):
    w = wl.frame1080(W=640, H=360, n_boxes=16, side_range=(12, 160))
    params = dict(w.params, dy_min=-2, dy_max=1, far_dmin=-3, far_dmax=28, close_dmin=-4,
                  close_dmax=50, grid_g=3, agg_nmin=3)
    got, ref, _, nc = _run_frame(torch_cuda, w, params=params)
    compare_box_outputs(got, ref, "dy")
    compare_debug(got["debug"], ref, nc, "dy")


def test_trimmed_mean_grid5(torch_cuda):
    w = wl.batch8x2160(n_frames=1, W=1280, H=720, n_boxes=40, side_range=(12, 400))
    got, ref, _, nc = _run_frame(torch_cuda, w)
    compare_box_outputs(got, ref, "trim")
    compare_debug(got["debug"], ref, nc, "trim")


def test_census_5x5_k3_sentinel0(torch_cuda):
    w = wl.frame1080(W=500, H=300, n_boxes=20, side_range=(12, 200))
    params = dict(w.params, win_w=5, win_h=5, sentinel=0, close_factor=3, close_dmax=40)
    got, ref, _, nc = _run_frame(torch_cuda, w, params=params)
    compare_box_outputs(got, ref, "5x5k3")
    compare_debug(got["debug"], ref, nc, "5x5k3")


def test_zero_boxes_and_capacity(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    w = wl.frame1080(W=320, H=200, n_boxes=6, side_range=(12, 80))
    fr = w.frames[0]
    ctx = B.Context(w.params, 1, 320, 200, 6)
    L, R = torch_frames([fr])[0]
    empty = torch_cuda.zeros((0, 5), dtype=torch_cuda.int32, device="cuda")
    out = ctx.match_boxes(L, R, empty, fr.f_px, fr.baseline_m)
    torch_cuda.cuda.synchronize()
    assert out["disp"].numel() == 0
    assert ctx.stats()["n_blocks"] == 0
    bt = torch_cuda.from_numpy(np.ascontiguousarray(w.boxes)).cuda()
    got = ctx.match_boxes(L, R, bt, fr.f_px, fr.baseline_m)  # exactly at capacity
    ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    compare_box_outputs({k: v.cpu().numpy() for k, v in got.items()}, ref, "cap")
    with pytest.raises(B.CtmError):
        ctx.match_boxes(L, R, torch_cuda.cat([bt, bt]), fr.f_px, fr.baseline_m)  # beyond capacity
    big = torch_cuda.zeros((201, 320), dtype=torch_cuda.uint8, device="cuda")
    with pytest.raises(B.CtmError):
        ctx.match_boxes(big, big, bt, fr.f_px, fr.baseline_m)
    ctx.close()


def test_batch_graph_mixed_sizes(torch_cuda):
    """Frames of different sizes and box counts in one planned launch, replayed
    from the captured graph; equal to the oracle frame by frame."""
    from paper_2604_07980_gb300 import binding as B
    ws = [wl.frame1080(seed=3000 + i, W=W, H=H, n_boxes=nb, side_range=(12, 180))
          for i, (W, H, nb) in enumerate([(640, 360, 20), (800, 450, 0), (480, 300, 33), (960, 540, 12)])]
    frames = [f for w in ws for f in w.frames]
    boxes = np.concatenate([np.c_[w.boxes[:, :4], np.full(len(w.boxes), i)] for i, w in enumerate(ws)]
                           ).astype(np.int32).reshape(-1, 5)
    params = ws[0].params
    ctx = B.Context(params, 6, 960, 540, 100)
    batch = B.DeviceBatch(torch_frames(frames), boxes, [(f.f_px, f.baseline_m) for f in frames])
    outs = []
    for _ in range(3):
        got = ctx.match_batch(batch, use_graph=True, debug=True)
        torch_cuda.cuda.synchronize()
        outs.append({k: (v.cpu().numpy() if k != "debug" else v) for k, v in got.items()})
    ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in frames], boxes,
                          orc.Params(**params), debug=True)
    for o in outs:
        compare_box_outputs(o, ref, "batch")
        compare_debug(o["debug"], ref, B.n_candidates(ctx.params), "batch")
    nograph = ctx.match_batch(batch, use_graph=False)
    torch_cuda.cuda.synchronize()
    compare_box_outputs({k: v.cpu().numpy() for k, v in nograph.items()}, ref, "batch-nograph")
    assert ctx.stats()["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params)
    # host end-to-end entry point
    host = ctx.match_batch_host([(f.left, f.right) for f in frames], boxes,
                                [f.f_px for f in frames], [f.baseline_m for f in frames])
    compare_box_outputs(host, ref, "batch-host")
    ctx.close()


def test_batch_replay_with_fewer_frames(torch_cuda):
    """Counts live in device memory: the same graph replays with a smaller batch."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=3, W=640, H=400, mean_boxes=10, side_range=(12, 200))
    ctx = B.Context(w.params, 3, 640, 400, 200)
    batch = B.DeviceBatch(torch_frames(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    ctx.match_batch(batch, use_graph=True)
    n0 = int((w.boxes[:, 4] == 0).sum())
    batch.counts.copy_(torch_cuda.tensor([1, n0], dtype=torch_cuda.int32))
    batch.disp.fill_(-7.0)
    got = ctx.match_batch(batch, use_graph=True)
    torch_cuda.cuda.synchronize()
    fr = w.frames[0]
    ref = orc.match_frame(fr.left, fr.right, w.boxes[:n0], fr.f_px, fr.baseline_m, orc.Params(**w.params))
    compare_box_outputs({k: v.cpu().numpy()[:n0] for k, v in got.items()}, ref, "replay")
    assert np.all(batch.disp.cpu().numpy()[n0:len(w.boxes)] == -7.0)
    ctx.close()


def test_batch_host_merged_copies(torch_cuda):
    """Host batch whose images are packed at the staging pitch and laid out back to back
    (one merged copy), and the same images in an order that breaks the runs (several
    copies): both equal the oracle."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=4, W=1024, H=256, mean_boxes=8, side_range=(12, 160))
    ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                          orc.Params(**w.params))
    ctx = B.Context(w.params, 4, 1024, 256, w.n_boxes)
    packed = np.empty((4, 2, 256, 1024), np.uint8)
    for i, f in enumerate(w.frames):
        packed[i, 0], packed[i, 1] = f.left, f.right
    fpx = [f.f_px for f in w.frames]
    bm = [f.baseline_m for f in w.frames]
    got = ctx.match_batch_host([(packed[i, 0], packed[i, 1]) for i in range(4)], w.boxes, fpx, bm)
    compare_box_outputs(got, ref, "host, one merged copy")
    swapped = np.empty_like(packed)  # right image first in memory: no run continues
    swapped[:, 0], swapped[:, 1] = packed[:, 1], packed[:, 0]
    got = ctx.match_batch_host([(swapped[i, 1], swapped[i, 0]) for i in range(4)], w.boxes, fpx, bm)
    compare_box_outputs(got, ref, "host, separate copies")
    got = ctx.match_batch_host_packed(packed, w.boxes, fpx, bm)
    compare_box_outputs(got, ref, "host, packed array")
    ctx.close()


def test_batch_host_sub_batches_equal_device_batch(torch_cuda):
    """The host entry point splits chained frames into sub-batches whose copies
    overlap the previous sub-batch's kernels: outputs and summed counters equal the
    one-launch device path bit for bit.  Boxes listed out of frame order are not
    chained and run as one batch, with the same outputs."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=7, W=800, H=400, mean_boxes=10, side_range=(12, 200))
    ctx = B.Context(w.params, 7, 800, 400, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    dev = ctx.match_batch(batch, use_graph=True)
    torch_cuda.cuda.synchronize()
    dev = {k: v.cpu().numpy() for k, v in dev.items()}
    st_dev = ctx.stats()
    fpx = [f.f_px for f in w.frames]
    bm = [f.baseline_m for f in w.frames]
    host = ctx.match_batch_host([(f.left, f.right) for f in w.frames], w.boxes, fpx, bm)
    st_host = ctx.stats()
    for k in ("disp", "depth", "flags"):
        assert np.array_equal(host[k], dev[k], equal_nan=True), k
    for k in ("cost_evals", "n_blocks", "n_boxes", "census_tiles", "error"):
        assert st_host[k] == st_dev[k], (k, st_host[k], st_dev[k])
    ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                          orc.Params(**w.params))
    compare_box_outputs(host, ref, "host sub-batches")
    # frame 0's boxes listed after all others: not chained, one batch
    counts = np.bincount(w.boxes[:, 4], minlength=7)
    order = np.concatenate([np.nonzero(w.boxes[:, 4] != 0)[0], np.nonzero(w.boxes[:, 4] == 0)[0]])
    bx = np.ascontiguousarray(w.boxes[order], dtype=np.int32)
    begins = np.zeros(7, np.int64)
    begins[1:] = np.concatenate([[0], np.cumsum(counts[1:])[:-1]])
    begins[0] = counts[1:].sum()
    arr = (B.ctm_frame * 7)()
    for i, f in enumerate(w.frames):
        arr[i] = B.ctm_frame(f.left.ctypes.data, f.right.ctypes.data, 800, 400, f.left.strides[0],
                             int(begins[i]), int(counts[i]), float(f.f_px), float(f.baseline_m))
    n = len(bx)
    disp = np.empty(n, np.float32)
    depth = np.empty(n, np.float32)
    flags = np.empty(n, np.uint8)
    assert B.lib().ctm_match_batch_host(ctx._h, arr, 7, bx.ctypes.data, n, disp.ctypes.data,
                                        depth.ctypes.data, flags.ctypes.data, None) == B.CTM_OK
    assert np.array_equal(flags, dev["flags"][order])
    assert np.array_equal(disp, dev["disp"][order], equal_nan=True)
    assert np.array_equal(depth, dev["depth"][order], equal_nan=True)
    assert ctx.stats()["cost_evals"] == st_dev["cost_evals"]
    ctx.close()


@pytest.mark.parametrize("n_ctx", [2, 3])
def test_contexts_in_flight_on_their_own_streams(torch_cuda, n_ctx):
    """Contexts replaying their graphs round robin on streams of their own (the
    benchmark's batches in flight) give the same outputs and counters as one context
    alone."""
    from paper_2604_07980_gb300 import binding as B
    torch = torch_cuda
    w = wl.batch32x1200(n_frames=6, W=960, H=600, mean_boxes=12, side_range=(12, 240))
    frames = B.frames_to_device(w.frames)
    calib = [(f.f_px, f.baseline_m) for f in w.frames]
    ctxs = [B.Context(w.params, 6, 960, 600, w.n_boxes) for _ in range(n_ctx)]
    batches = [B.DeviceBatch(frames, w.boxes, calib) for _ in range(n_ctx)]
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream() for _ in range(n_ctx - 1)]
    ref = ctxs[0].match_batch(batches[0], use_graph=True)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy().copy() for k, v in ref.items()}
    st_ref = ctxs[0].stats()
    for i in range(4 * n_ctx):
        ctxs[i % n_ctx].match_batch(batches[i % n_ctx], use_graph=True, stream=streams[i % n_ctx])
    torch.cuda.synchronize()
    for c, b in zip(ctxs, batches):
        assert c.stats()["cost_evals"] == st_ref["cost_evals"] and c.stats()["error"] == 0
        for k in ("disp", "depth", "flags"):
            got = getattr(b, k)[:b.n_boxes].cpu().numpy()
            assert np.array_equal(got, ref[k], equal_nan=True), k
    oref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                           orc.Params(**w.params))
    compare_box_outputs(ref, oref, f"{n_ctx} contexts")
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("n_boxes", [300, 1100])
def test_many_boxes_in_one_frame(torch_cuda, n_boxes):
    """Frames with more boxes than the planner keeps in registers (256 per warp's
    lanes) and than it stages in shared memory (1024): the occluder selection falls
    back to scanning the frame's boxes from shared or global memory; equal to the
    oracle, block records included."""
    w = wl.frame1080(W=800, H=600, n_boxes=n_boxes, side_range=(8, 90), seed=4100 + n_boxes)
    params = dict(w.params, max_occluders=16, frontal_crop=0.3)
    got, ref, stats, nc = _run_frame(torch_cuda, w, params=params)
    compare_box_outputs(got, ref, f"{n_boxes} boxes")
    compare_debug(got["debug"], ref, nc, f"{n_boxes} boxes")
    assert stats["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], params)


def test_frontal_crop_occluder_priority(torch_cuda):
    """Occluder cap of 2 with the frontal-crop priority on a batch with many overlapping
    boxes: block records and outputs equal the oracle's (and differ from proximity-only
    ranking somewhere, so the rule is exercised)."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=3)
    params = dict(w.params, max_occluders=2, frontal_crop=0.4)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**params), debug=True)
    near = orc.match_batch(frames, w.boxes, orc.Params(**dict(params, frontal_crop=0.0)), debug=True)
    assert not np.array_equal(ref["blocks"]["n_valid"], near["blocks"]["n_valid"])
    ctx = B.Context(params, len(w.frames), 1920, 1200, w.n_boxes)
    batch = B.DeviceBatch(torch_frames(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    got = ctx.match_batch(batch, use_graph=True, debug=True)
    torch_cuda.cuda.synchronize()
    compare_box_outputs({k: v.cpu().numpy() for k, v in got.items() if k != "debug"}, ref, "frontal crop")
    compare_debug(got["debug"], ref, B.n_candidates(ctx.params), "frontal crop")
    ctx.close()


@pytest.mark.parametrize("name", ["pair640", "frame1080", "batch32x1200", "batch8x2160"])
def test_disparity_chunk_tiles_bit_exact(torch_cuda, name):
    """(block, disparity-chunk) tiles of the fused matcher: forced 2, 4 and 8 ways,
    the automatic choice and no splitting all give the oracle's block records, every
    forward and backward cost, box outputs and evaluation count (ties included: the
    chunk minima merge as (cost, candidate) keys)."""
    from paper_2604_07980_gb300 import binding as B
    if name == "batch32x1200":
        w = wl.batch32x1200(n_frames=3)
    elif name == "batch8x2160":
        w = wl.batch8x2160(n_frames=1, n_boxes=48)
    else:
        w = wl.by_name(name)
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**w.params), debug=True)
    H, W = w.frames[0].left.shape
    ctx = B.Context(w.params, len(w.frames), W, H, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    for ways in (0, 1, 2, 4, 8):
        ctx.set_tuning(split_ways=ways)
        for graph in (False, True):
            got = ctx.match_batch(batch, use_graph=graph, debug=True)
            torch_cuda.cuda.synchronize()
            where = f"{name} split_ways {ways} graph {graph}"
            out = {k: v.cpu().numpy() for k, v in got.items() if k != "debug"}
            compare_box_outputs(out, ref, where)
            compare_debug(got["debug"], ref, B.n_candidates(ctx.params), where)
            st = ctx.stats()
            assert st["error"] == 0, where
            assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params), where
    ctx.close()


@pytest.mark.parametrize("threads,strip_extra", [(128, 0), (256, 0), (256, 320)])
def test_queue_rounds_bit_exact(torch_cuda, threads, strip_extra):
    """Per-SM rounds over the work-ordered queue (a context whose capacity fits in
    the rounds, so the rounds variant of the persistent matcher runs) against the
    oracle and against one dynamic queue: block records, every cost, box outputs and
    the evaluation count.  With 256 threads and a wide strip only three CTAs fit an
    SM, so the fourth round has no CTA of its rank anywhere and every one of its
    positions is swept up by CTAs asking for their next block."""
    from paper_2604_07980_gb300 import binding as B
    sms = torch_cuda.cuda.get_device_properties(0).multi_processor_count
    w = wl.frame1080()
    slots = w.params.get("grid_g", 4) ** 2
    if w.n_boxes * slots > 8 * sms:
        pytest.skip("the context's capacity does not fit in the rounds on this GPU")
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**w.params), debug=True)
    H, W = w.frames[0].left.shape
    ctx = B.Context(w.params, len(w.frames), W, H, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    cols = ctx.get_tuning()["strip_cols"] + strip_extra
    for rounds in (1, 0):
        ctx.set_tuning(match_threads=threads, strip_cols=cols, split_ways=1, queue_rounds=rounds)
        for graph in (False, True):
            got = ctx.match_batch(batch, use_graph=graph, debug=True)
            torch_cuda.cuda.synchronize()
            where = f"threads {threads} strip {cols} rounds {rounds} graph {graph}"
            out = {k: v.cpu().numpy() for k, v in got.items() if k != "debug"}
            compare_box_outputs(out, ref, where)
            compare_debug(got["debug"], ref, B.n_candidates(ctx.params), where)
            st = ctx.stats()
            assert st["error"] == 0, where
            assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params), where
    ctx.close()
