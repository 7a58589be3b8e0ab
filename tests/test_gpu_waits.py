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
