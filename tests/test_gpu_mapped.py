"""ctm_match_batch_mapped: the device reads, straight from host memory, only the
image bytes the census of the marked tiles needs.  Outputs must equal the oracle
and the copying host path bit for bit (integer outputs; disparity within 1e-4 px,
depth within 1e-5 relative), with the staging images holding other images' bytes
beforehand, so that a census read outside the gathered bytes would show.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl
from tests.parity_util import compare_box_outputs, oracle_evals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _workload(name):
    if name == "batch32x1200":
        return wl.batch32x1200(n_frames=3)
    if name == "batch8x2160":
        return wl.batch8x2160(n_frames=1, n_boxes=48)
    return wl.by_name(name)


def _pinned(torch, arrays):
    t = torch.empty(arrays.shape, dtype=torch.uint8, pin_memory=True)
    a = t.numpy()
    a[...] = arrays
    return t, a


@pytest.mark.parametrize("name", ["pair640", "frame1080", "batch32x1200", "batch8x2160"])
def test_mapped_equals_oracle_and_copy_path(torch_cuda, name):
    from paper_2604_07980_gb300 import binding as B
    w = _workload(name)
    nf = len(w.frames)
    H, W = w.frames[0].left.shape
    frames = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames]
    ref = orc.match_batch(frames, w.boxes, orc.Params(**w.params), debug=True)
    fpx = [f.f_px for f in w.frames]
    bm = [f.baseline_m for f in w.frames]
    packed = np.stack([np.stack([f.left, f.right]) for f in w.frames])
    keep, images = _pinned(torch_cuda, packed)
    noise = np.random.default_rng(7).integers(0, 256, packed.shape, dtype=np.uint8)
    keep_n, noise_p = _pinned(torch_cuda, noise)
    ctx = B.Context(w.params, nf, W, H, w.n_boxes)
    # staging images filled with noise by the copying path, then the mapped call
    ctx.match_batch_host_packed(noise_p, w.boxes, fpx, bm)
    got = ctx.match_batch_host_packed(images, w.boxes, fpx, bm, mapped=True)
    st = ctx.stats()
    compare_box_outputs(got, ref, f"{name} mapped")
    assert st["error"] == 0
    assert st["cost_evals"] == oracle_evals(ref["blocks"], ref["flags"], w.params)
    assert 0 < st["host_bytes"] <= packed.nbytes, st["host_bytes"]
    got = {k: v.copy() for k, v in got.items()}
    # the same call through the per-frame table, then the copying path
    again = ctx.match_batch_host([(images[i, 0], images[i, 1]) for i in range(nf)], w.boxes, fpx, bm, mapped=True)
    assert ctx.stats()["host_bytes"] == st["host_bytes"]
    copied = ctx.match_batch_host_packed(images, w.boxes, fpx, bm)
    assert ctx.stats()["host_bytes"] == 0
    for k in ("disp", "depth", "flags"):
        assert np.array_equal(again[k], got[k], equal_nan=True), k
        assert np.array_equal(copied[k], got[k], equal_nan=True), k
    ctx.close()


def test_mapped_pageable_memory(torch_cuda):
    """Plain (pageable) numpy images: read in place where the device has pageable
    memory access, else copied whole (no bytes read in place); outputs equal the
    oracle's either way."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.frame1080()
    fr = w.frames[0]
    H, W = fr.left.shape
    ref = orc.match_frame(fr.left, fr.right, w.boxes, fr.f_px, fr.baseline_m, orc.Params(**w.params))
    ctx = B.Context(w.params, 1, W, H, w.n_boxes)
    left, right = np.ascontiguousarray(fr.left), np.ascontiguousarray(fr.right)
    assert left.ctypes.data % 16 == 0 and right.ctypes.data % 16 == 0
    got = ctx.match_batch_host([(left, right)], w.boxes, fr.f_px, fr.baseline_m, mapped=True)
    compare_box_outputs(got, ref, "mapped, pageable")
    ctx.close()


def test_mapped_unaligned_frames_copied(torch_cuda):
    """Frames whose rows or width are off 16-byte multiples are copied whole, beside
    frames read in place in the same call; outputs equal the oracle's."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=3, W=640, H=400, mean_boxes=10, side_range=(12, 200))
    H, W = w.frames[0].left.shape
    _, pinned = _pinned(torch_cuda, np.stack([np.stack([f.left, f.right]) for f in w.frames]))
    wide = np.zeros((3, 2, H, W + 8), np.uint8)  # frame 1 read from 4 bytes into its rows
    wide[1, :, :, 4:4 + W] = pinned[1]
    frames = [(pinned[0, 0], pinned[0, 1]), (wide[1, 0][:, 4:4 + W], wide[1, 1][:, 4:4 + W]),
              (pinned[2, 0], pinned[2, 1])]
    ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                          orc.Params(**w.params))
    ctx = B.Context(w.params, 3, W, H, w.n_boxes)
    got = ctx.match_batch_host(frames, w.boxes, [f.f_px for f in w.frames], [f.baseline_m for f in w.frames],
                               mapped=True)
    compare_box_outputs(got, ref, "mapped with an unaligned frame")
    assert 0 < ctx.stats()["host_bytes"]
    narrow = ctx.match_batch_host([(f.left[:, :632], f.right[:, :632]) for f in w.frames[:1]],
                                  w.boxes[w.boxes[:, 4] == 0], w.frames[0].f_px, w.frames[0].baseline_m,
                                  mapped=True)
    ref0 = orc.match_frame(np.ascontiguousarray(w.frames[0].left[:, :632]),
                           np.ascontiguousarray(w.frames[0].right[:, :632]), w.boxes[w.boxes[:, 4] == 0],
                           w.frames[0].f_px, w.frames[0].baseline_m, orc.Params(**w.params))
    compare_box_outputs(narrow, ref0, "mapped, width 632 (copied)")
    assert ctx.stats()["host_bytes"] == 0
    ctx.close()
