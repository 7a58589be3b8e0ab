"""Host-side fault injection: device allocations that fail (as cudaMalloc does on
an exhausted device) make context creation, the host-buffer entry point's
staging and server creation return CTM_ENOMEM, release everything they had
allocated (the device's free memory returns to where it was), and leave the
library usable: the next calls succeed and match the oracle.  No GPU fault is
involved; the failure is made on the host."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _free(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_context_and_host_staging_allocation_failures(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    w = wl.pair640()
    fr = w.frames[0]
    free0 = _free(torch_cuda)
    assert L.ctm_inject_alloc_failures(0, 1) == B.CTM_OK
    with pytest.raises(B.CtmError) as ei:
        B.Context(w.params, 1, 640, 480, len(w.boxes))
    assert ei.value.status == B.CTM_ENOMEM
    assert _free(torch_cuda) == free0
    ctx = B.Context(w.params, 1, 640, 480, len(w.boxes))  # the injection was consumed
    ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    assert L.ctm_inject_alloc_failures(0, 1) == B.CTM_OK
    with pytest.raises(B.CtmError) as ei:
        ctx.match_batch_host([(fr.left, fr.right)], w.boxes, fr.f_px, fr.baseline_m)
    assert ei.value.status == B.CTM_ENOMEM
    host = ctx.match_batch_host([(fr.left, fr.right)], w.boxes, fr.f_px, fr.baseline_m)
    compare_box_outputs(host, ref, "host path after a failed staging allocation")
    ctx.close()
    assert L.ctm_inject_alloc_failures(-1, 1) == B.CTM_EINVAL
    assert L.ctm_inject_alloc_failures(0, 0) == B.CTM_OK


def test_server_creation_allocation_failures(torch_cuda):
    """Server creation makes five device allocations with two lanes (the arena, then
    per lane its context workspace and its batch buffers); each one failing in turn
    gives CTM_ENOMEM with nothing left allocated, and then a server serves a frame."""
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    w = wl.pair640()
    fr = w.frames[0]
    cfg = dict(lanes=2, frames_per_batch=2, max_width=640, max_height=480, max_boxes_per_frame=8,
               max_queue=8, image_budget_bytes=8 << 20)
    B.Server(w.params, **cfg).close()  # the driver's one-time state (graph instantiation) first
    free0 = _free(torch_cuda)
    for k in range(5):
        assert L.ctm_inject_alloc_failures(k, 1) == B.CTM_OK
        with pytest.raises(B.CtmError) as ei:
            B.Server(w.params, **cfg)
        assert ei.value.status == B.CTM_ENOMEM, k
        assert _free(torch_cuda) == free0, f"allocation {k} failing leaked device memory"
    assert L.ctm_inject_alloc_failures(0, 0) == B.CTM_OK
    srv = B.Server(w.params, **cfg)
    Lp = torch_cuda.from_numpy(fr.left).pin_memory()
    Rp = torch_cuda.from_numpy(fr.right).pin_memory()
    tag = srv.submit(Lp, Rp, w.boxes, fr.f_px, fr.baseline_m)
    assert tag is not None
    done = srv.wait_all()
    assert len(done) == 1 and done[0]["status"] == 0
    ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    compare_box_outputs(done[0], ref, "served after failed creations")
    srv.close()
