"""A bounded device wait that runs out (an mbarrier phase that nothing
completes, waited on with the matching kernels' own routine) ends its kernel
with the expiry recorded in a device flag, and the context stays usable: a
match call afterwards gives the oracle's outputs and no error."""
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_context_stays_usable():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    w = wl.pair640()
    fr = w.frames[0]
    ctx = B.Context(w.params, 1, 640, 480, len(w.boxes))
    expired, ms = B.probe_bounded_wait()
    assert expired == 1
    assert 500.0 < ms < 10000.0  # two waits of about one second each
    L = torch.from_numpy(fr.left).cuda()
    R = torch.from_numpy(fr.right).cuda()
    got = ctx.match_boxes(L, R, torch.from_numpy(w.boxes).cuda(), fr.f_px, fr.baseline_m)
    torch.cuda.synchronize()
    assert ctx.stats()["error"] == 0
    ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    compare_box_outputs({k: v.cpu().numpy() for k, v in got.items()}, ref, "after an expired wait")
    host = ctx.match_batch_host([(fr.left, fr.right)], w.boxes, fr.f_px, fr.baseline_m)  # CTM_OK
    compare_box_outputs(host, ref, "host path after an expired wait")
    ctx.close()


def test_matcher_wait_expiry_invalidates_every_searched_box():
    """The matcher's own bounded wait (Sec. 4.3.3: an unverified match must not
    be reported).  The test-only injection makes the first matching CTA announce
    a strip copy on its mbarrier without issuing it; its wait expires, it stops,
    and the other CTAs finish the queue.  Every box that needed a search must
    then come out with flags 0 and NaN outputs (its blocks may be stale), boxes
    without blocks keep their planner outputs, the device flag and the host
    entry point's status report the expiry, and the next call equals the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import numpy as np

    from paper_2604_07980_gb300 import binding as B
    w = wl.frame1080()
    fr = w.frames[0]
    H, W = fr.left.shape
    # the frame's 64 boxes plus two that are empty after clipping (no blocks)
    boxes = np.concatenate([w.boxes, np.array([[W + 10, 10, W + 50, 50, 0], [100, 100, 100, 140, 0]],
                                              np.int32)]).astype(np.int32)
    n = len(boxes)
    ctx = B.Context(w.params, 1, W, H, n)
    L = torch.from_numpy(fr.left).cuda()
    R = torch.from_numpy(fr.right).cuda()
    bt = torch.from_numpy(boxes).cuda()
    ref = orc.match_frame(fr.left, fr.right, boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    searched = (ref["flags"] & orc.BOX_EMPTY) == 0
    assert searched.sum() > 10 and (~searched).sum() > 0  # both kinds occur in this frame

    def check_invalidated(got, where):
        gf = np.asarray(got["flags"]).astype(np.uint8)
        assert np.all(gf[searched] == 0), f"{where}: searched boxes keep flags {gf[searched][:8]}"
        assert np.all(np.isnan(np.asarray(got["disp"])[searched])), where
        assert np.all(np.isnan(np.asarray(got["depth"])[searched])), where
        sub = {k: np.asarray(v)[~searched] for k, v in got.items()}
        compare_box_outputs(sub, {k: np.asarray(v)[~searched] for k, v in ref.items()
                                  if k in ("flags", "disp", "depth")}, f"{where}, boxes without blocks")

    # device entry point: the flag is left in ctm_stats.error
    ctx.inject_wait_expiry()
    got = ctx.match_boxes(L, R, bt, fr.f_px, fr.baseline_m)
    torch.cuda.synchronize()
    assert ctx.stats()["error"] != 0
    check_invalidated({k: v.cpu().numpy() for k, v in got.items()}, "device call after expiry")

    # the next call is clean and equals the oracle
    got = ctx.match_boxes(L, R, bt, fr.f_px, fr.baseline_m)
    torch.cuda.synchronize()
    assert ctx.stats()["error"] == 0
    compare_box_outputs({k: v.cpu().numpy() for k, v in got.items()}, ref, "device call after recovery")

    # host entry point: the status is CTM_ETIMEOUT and the outputs are invalidated too
    ctx.inject_wait_expiry()
    out = (np.full(n, 7.0, np.float32), np.full(n, 7.0, np.float32), np.full(n, 0xff, np.uint8))
    with pytest.raises(B.CtmError) as ei:
        ctx.match_batch_host([(fr.left, fr.right)], boxes, fr.f_px, fr.baseline_m, out=out)
    assert ei.value.status == B.CTM_ETIMEOUT
    check_invalidated({"disp": out[0], "depth": out[1], "flags": out[2]}, "host call after expiry")
    host = ctx.match_batch_host([(fr.left, fr.right)], boxes, fr.f_px, fr.baseline_m)
    compare_box_outputs(host, ref, "host call after recovery")
    ctx.close()
