"""ctm_match_boxes_noalloc: the entry point for callers that cannot call
cudaMalloc while they run (real-time loops, where an allocation can synchronize
the device and take an unbounded time; hosts that give the library a fixed
memory budget up front).  Called through the C ABI, it must give the results of
the ordinary context path on consecutive calls -- different frames and
parameters, then the first again -- although every call reuses the same static
device workspace; it must not change the device's free memory; and its counters
(ctm_noalloc_get_stats) must report the call's evaluations and no expired wait.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _inputs(torch, w):
    fr = w.frames[0]
    L = torch.from_numpy(np.ascontiguousarray(fr.left)).cuda()
    R = torch.from_numpy(np.ascontiguousarray(fr.right)).cuda()
    boxes = torch.from_numpy(np.ascontiguousarray(w.boxes)).cuda()
    return fr, L, R, boxes


def _noalloc(torch, B, w, L, R, boxes, fr):
    n = int(boxes.shape[0])
    p = B.make_params(w.params)
    disp = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    depth = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    flags = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    H, W = L.shape
    st = B.lib().ctm_match_boxes_noalloc(
        ctypes.byref(p), ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(R.data_ptr()), W, H,
        L.stride(0), ctypes.c_void_p(boxes.data_ptr()), n, fr.f_px, fr.baseline_m,
        ctypes.c_void_p(disp.data_ptr()), ctypes.c_void_p(depth.data_ptr()),
        ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.CTM_OK, B.lib().ctm_status_str(st)
    torch.cuda.synchronize()
    return {"disp": disp.cpu().numpy(), "depth": depth.cpu().numpy(), "flags": flags.cpu().numpy()}


def _context(torch, B, w, L, R, boxes, fr):
    H, W = L.shape
    ctx = B.Context(w.params, 1, W, H, max(int(boxes.shape[0]), 1))
    out = ctx.match_boxes(L, R, boxes, fr.f_px, fr.baseline_m)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = ctx.stats()
    ctx.close()
    return res


def _noalloc_stats(B):
    s = B.ctm_stats()
    st = B.lib().ctm_noalloc_get_stats(ctypes.byref(s), None)
    assert st == B.CTM_OK, B.lib().ctm_status_str(st)
    return {"cost_evals": int(s.cost_evals), "n_boxes": int(s.n_boxes), "error": int(s.error)}


def test_noalloc_equals_context_path_on_consecutive_calls(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    wa = wl.pair640()
    wb = wl.frame1080(W=640, H=480, n_boxes=48, side_range=(12, 200))
    runs = []
    for w in (wa, wb, wa):
        fr, L, R, boxes = _inputs(torch_cuda, w)
        ref = _context(torch_cuda, B, w, L, R, boxes, fr)
        got = _noalloc(torch_cuda, B, w, L, R, boxes, fr)
        compare_box_outputs(got, ref, f"noalloc {w.name}")
        st = _noalloc_stats(B)
        assert st["error"] == 0
        assert st["cost_evals"] == ref["stats"]["cost_evals"] > 0
        assert st["n_boxes"] == len(w.boxes)
        runs.append(got)
    assert np.array_equal(runs[0]["flags"], runs[2]["flags"])
    assert np.array_equal(runs[0]["disp"], runs[2]["disp"], equal_nan=True)


def test_noalloc_leaves_device_free_memory_unchanged(torch_cuda):
    """Every buffer is made before the first call; after a warm-up call, calls with
    other frames and parameters must not change the device's free memory."""
    from paper_2604_07980_gb300 import binding as B
    torch = torch_cuda
    ws = [wl.pair640(), wl.frame1080(W=640, H=480, n_boxes=48, side_range=(12, 200))]
    ws.append(wl.frame1080(W=320, H=200, n_boxes=9, side_range=(12, 120)))
    ws[2].params = dict(ws[2].params, win_w=5, win_h=5, close_factor=3, grid_g=3, agg_nmin=3)
    staged = []
    for w in ws:
        fr, L, R, boxes = _inputs(torch, w)
        n = int(boxes.shape[0])
        outs = (torch.empty(n, dtype=torch.float32, device="cuda"),
                torch.empty(n, dtype=torch.float32, device="cuda"),
                torch.empty(n, dtype=torch.uint8, device="cuda"))
        staged.append((B.make_params(w.params), fr, L, R, boxes, n, outs))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(i):
        p, fr, L, R, boxes, n, (disp, depth, flags) = staged[i]
        H, W = L.shape
        st = B.lib().ctm_match_boxes_noalloc(
            ctypes.byref(p), ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(R.data_ptr()), W, H,
            L.stride(0), ctypes.c_void_p(boxes.data_ptr()), n, fr.f_px, fr.baseline_m,
            ctypes.c_void_p(disp.data_ptr()), ctypes.c_void_p(depth.data_ptr()),
            ctypes.c_void_p(flags.data_ptr()), stream)
        assert st == B.CTM_OK, B.lib().ctm_status_str(st)

    call(0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in (1, 2, 0, 2, 1):
        call(i)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_limits(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    w = wl.pair640()
    fr, L, R, boxes = _inputs(torch_cuda, w)
    big = torch_cuda.zeros((481, 640), dtype=torch_cuda.uint8, device="cuda")
    p = B.make_params(w.params)
    out = torch_cuda.empty(4, dtype=torch_cuda.float32, device="cuda")
    fl = torch_cuda.empty(4, dtype=torch_cuda.uint8, device="cuda")
    st = B.lib().ctm_match_boxes_noalloc(
        ctypes.byref(p), ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()), 640, 481, 640,
        ctypes.c_void_p(boxes.data_ptr()), 4, fr.f_px, fr.baseline_m, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(fl.data_ptr()), None)
    assert st == B.CTM_ETOOBIG
    many = torch_cuda.zeros((65, 5), dtype=torch_cuda.int32, device="cuda")
    st = B.lib().ctm_match_boxes_noalloc(
        ctypes.byref(p), ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(R.data_ptr()), 640, 480, 640,
        ctypes.c_void_p(many.data_ptr()), 65, fr.f_px, fr.baseline_m, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(fl.data_ptr()), None)
    assert st == B.CTM_ETOOBIG


def test_noalloc_random_configurations_equal_oracle(torch_cuda):
    """The seeded random parameter sets of the GPU parity sweep, first frame of each,
    through the allocation-free entry point: equal to the oracle."""
    from oracle import oracle as orc
    from paper_2604_07980_gb300 import binding as B
    from tests.test_gpu_random_configs import _random_params
    ran = 0
    for seed in range(40):
        rng = np.random.default_rng(7000 + seed)
        params = _random_params(rng)
        n_frames = int(rng.integers(1, 4))
        W, H = int(rng.integers(60, 260)), int(rng.integers(50, 200))
        w = wl.multi_frame("frame1080", 8000 + seed, n_frames, W, H, int(rng.integers(3, 25)), (4.0, 120.0),
                           (0.5, 12.0), (1.0, 24.0), strip_frac=0.3)
        w.params = params
        sel = w.boxes[:, 4] == 0
        w.boxes = np.ascontiguousarray(w.boxes[sel])
        if len(w.boxes) == 0:
            continue
        fr, L, R, boxes = _inputs(torch_cuda, w)
        got = _noalloc(torch_cuda, B, w, L, R, boxes, fr)
        ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**params))
        compare_box_outputs(got, ref, f"noalloc seed {seed} params {params}")
        ran += 1
    assert ran >= 35
