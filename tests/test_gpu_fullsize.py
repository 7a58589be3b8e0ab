"""Parity at full workload sizes, in the launch configuration the benchmark
times (one captured-graph ctm_match_batch over the whole batch), against the
oracle on sampled frames (the oracle finishes a frame in about a second)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs, compare_debug_arrays, oracle_evals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _run_batch(torch, w, debug):
    from paper_2604_07980_gb300 import binding as B
    H, W = w.frames[0].left.shape
    ctx = B.Context(w.params, len(w.frames), W, H, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes,
                          [(f.f_px, f.baseline_m) for f in w.frames])
    ctx.match_batch(batch, use_graph=True)  # capture
    got = ctx.match_batch(batch, use_graph=True, debug=debug)  # replay
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if k != "debug" else v) for k, v in got.items()}
    stats = ctx.stats()
    return ctx, out, stats


def _check_frames(w, out, frames, nc):
    p = orc.Params(**w.params)
    blocks = out["debug"].blocks_np() if "debug" in out else None
    cf = out["debug"].cost_f.cpu().numpy() if "debug" in out else None
    cb = out["debug"].cost_b.cpu().numpy() if "debug" in out else None
    for fi in frames:
        sel = np.nonzero(w.boxes[:, 4] == fi)[0]
        fr = w.frames[fi]
        ref = orc.match_frame(fr.left, fr.right, w.boxes[sel], fr.f_px, fr.baseline_m, p, debug=True)
        got = {k: out[k][sel] for k in ("disp", "depth", "flags")}
        compare_box_outputs(got, ref, f"frame {fi}")
        if blocks is not None:
            compare_debug_arrays(blocks[sel], cf[sel], cb[sel], ref, nc, f"frame {fi}")


def test_batch32x1200_full_size(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200()
    ctx, out, stats = _run_batch(torch_cuda, w, debug=True)
    assert stats["error"] == 0
    assert stats["n_boxes"] == w.n_boxes
    _check_frames(w, out, [0, 9, 18, 31], B.n_candidates(ctx.params))
    # every box has been given flags (no stale outputs)
    assert np.all(out["flags"] != 0)
    ctx.close()


def test_batch8x2160_full_size(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch8x2160()
    ctx, out, stats = _run_batch(torch_cuda, w, debug=False)
    assert stats["error"] == 0
    _check_frames(w, out, [0, 5], B.n_candidates(ctx.params))
    ctx.close()


def test_batch32x1200_eval_count_matches_oracle(torch_cuda):
    """The device evaluation count (the benchmark's unit of work) equals the
    oracle's count on a 4-frame batch of the same workload."""
    w = wl.batch32x1200(n_frames=4)
    ctx, out, stats = _run_batch(torch_cuda, w, debug=False)
    ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                          orc.Params(**w.params), debug=True)
    assert stats["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params)
    compare_box_outputs(out, ref, "4-frame batch")
    ctx.close()
