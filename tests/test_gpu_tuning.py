"""The autotuner and explicit tunings change launch shapes only: every tuning
gives bit-identical outputs and evaluation counts on the same batch, and the
tuning the autotuner keeps is one of its candidates."""
import numpy as np
import pytest

from paper_2604_07980_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _outputs(torch, ctx, batch):
    got = ctx.match_batch(batch, use_graph=True)
    torch.cuda.synchronize()
    return ({k: v.cpu().numpy().copy() for k, v in got.items()}, ctx.stats())


def test_tunings_do_not_change_results(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=6)
    ctx = B.Context(w.params, len(w.frames), 1920, 1200, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    ref, st0 = _outputs(torch_cuda, ctx, batch)
    nd = max(w.params["far_dmax"] - w.params["far_dmin"], w.params["close_dmax"] - w.params["close_dmin"]) + 1
    base = ((nd + 34 + 31) // 32) * 32
    for matcher in (0, 1):
      for th in (128, 256):
        for cols in (base, base + 64, base + 192):
            for mode in (0, 1, 2):
                for split in (0, 1):
                    ctx.set_tuning(match_threads=th, strip_cols=cols, census_mode=mode, queue_rounds=split,
                                   match_mode=matcher)
                    out, st = _outputs(torch_cuda, ctx, batch)
                    where = f"matcher {matcher} threads {th} cols {cols} census {mode} rounds {split}"
                    assert st["cost_evals"] == st0["cost_evals"] and st["error"] == 0, where
                    assert np.array_equal(out["flags"], ref["flags"]), where
                    assert np.array_equal(out["disp"], ref["disp"], equal_nan=True), where
                    assert np.array_equal(out["depth"], ref["depth"], equal_nan=True), where
    best, ms = ctx.autotune(batch, reps=2)
    assert ms > 0 and best["match_threads"] in (128, 256) and best["census_mode"] in (0, 1, 2)
    assert best["match_mode"] in (0, 1)
    assert best["strip_cols"] % 32 == 0 and best["strip_cols"] >= nd + 2
    assert ctx.get_tuning() == best
    out, st = _outputs(torch_cuda, ctx, batch)
    assert np.array_equal(out["flags"], ref["flags"])
    assert np.array_equal(out["disp"], ref["disp"], equal_nan=True)
    with pytest.raises(B.CtmError):
        ctx.set_tuning(match_threads=64)
    with pytest.raises(B.CtmError):
        ctx.set_tuning(strip_cols=nd)  # narrower than one disparity range
    assert ctx.get_tuning() == best    # unchanged after a refused tuning
    ctx.close()


def test_pipelined_matcher_debug_records_equal_fused(torch_cuda):
    """Block records and every forward/backward cost of the two-pass matcher equal
    the fused matcher's (which the oracle parity tests cover), chunked blocks included."""
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=4)
    ctx = B.Context(w.params, len(w.frames), 1920, 1200, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    res = {}
    for matcher in (0, 1):
        for th in (128, 256):
            ctx.set_tuning(match_mode=matcher, match_threads=th, strip_cols=192)
            got = ctx.match_batch(batch, use_graph=(th == 128), debug=True)
            torch_cuda.cuda.synchronize()
            res[(matcher, th)] = (got["debug"].blocks_np(), got["debug"].cost_f.cpu().numpy(),
                                  got["debug"].cost_b.cpu().numpy(), got["disp"].cpu().numpy(),
                                  got["flags"].cpu().numpy(), ctx.stats())
    ref = res[(0, 128)]
    for key, r in res.items():
        assert np.array_equal(r[0], ref[0]), key
        assert np.array_equal(r[1], ref[1]), key
        assert np.array_equal(r[2], ref[2]), key
        assert np.array_equal(r[3], ref[3], equal_nan=True), key
        assert np.array_equal(r[4], ref[4]), key
        assert r[5]["cost_evals"] == ref[5]["cost_evals"] and r[5]["error"] == 0, key
    ctx.close()
