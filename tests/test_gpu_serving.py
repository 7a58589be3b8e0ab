"""The serving loop (ctm_server_*): every frame's outputs are the same whether it
ran alone or batched with others (bit-identical: the batch runs the same integer
search and the same float steps per box), admission waits for arena space,
a full queue refuses without queueing, and the plain per-box serving mode gives
the same outputs.  Frames of a small served trace are also checked against the
single-frame entry point and, for one frame, the oracle."""
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


@pytest.fixture(scope="module")
def trace():
    # three streams, one per frame size, two rendered frames each
    return wl.serving(seed=2024, n_streams=3, duration_s=0.1, unique_frames=2, mean_boxes=40.0,
                      stream_sizes=((1280, 720), (1920, 1080), (3840, 2160)))


def _pinned(torch, tr):
    return [[(torch.from_numpy(f.left).pin_memory(), torch.from_numpy(f.right).pin_memory())
             for f in s.frames] for s in tr.streams]


def _same(a, b, where):
    assert np.array_equal(a["flags"], b["flags"]), where
    assert np.array_equal(a["disp"], b["disp"], equal_nan=True), where
    assert np.array_equal(a["depth"], b["depth"], equal_nan=True), where


def _alone(srv, tr, pinned):
    out = {}
    for s, st in enumerate(tr.streams):
        for k, fr in enumerate(st.frames):
            L, R = pinned[s][k]
            tag = srv.submit(L, R, st.boxes[k], fr.f_px, fr.baseline_m)
            (res,) = srv.wait_all()
            assert res["tag"] == tag and res["status"] == 0 and res["batch_frames"] == 1
            out[(s, k)] = res
    return out


@pytest.mark.parametrize("lanes", [2, 4])
def test_serving_alone_equals_mix(torch_cuda, trace, lanes):
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    srv = B.Server(trace.params, lanes=lanes, frames_per_batch=4, image_budget_bytes=1 << 30)
    alone = _alone(srv, trace, pinned)
    # the same frames, three times over, submitted in one burst
    keys = [(s, k) for s in range(len(trace.streams)) for k in range(2)] * 3
    tags = {}
    for key in keys:
        s, k = key
        fr = trace.streams[s].frames[k]
        tags[srv.submit(*pinned[s][k], trace.streams[s].boxes[k], fr.f_px, fr.baseline_m)] = key
    done = srv.wait_all()
    assert len(done) == len(keys)
    for r in done:
        assert r["status"] == 0
        _same(r, alone[tags[r["tag"]]], f"frame {tags[r['tag']]} in the mix")
    st = srv.stats()
    assert st["completed"] == st["submitted"] == len(alone) + len(keys)
    assert 2 <= st["max_lanes_busy"] <= lanes              # batches overlapped on the device
    assert st["batched_frames"] == st["completed"]
    assert st["batches"] < st["completed"]                 # frames were batched together
    assert max(r["batch_frames"] for r in done) > 1
    assert st["arena_peak_bytes"] <= st["arena_bytes"]
    for r in done:
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_launch_ns"] <= r["t_done_ns"]
    srv.close()

    # the served outputs equal the single-frame entry point's
    H, W = 2160, 3840
    ctx = B.Context(trace.params, 1, W, H, 256)
    for (s, k), r in alone.items():
        st_ = trace.streams[s]
        L, R = (t.cuda() for t in pinned[s][k])
        bx = torch_cuda.from_numpy(st_.boxes[k]).cuda()
        got = ctx.match_boxes(L, R, bx, st_.frames[k].f_px, st_.frames[k].baseline_m)
        torch_cuda.cuda.synchronize()
        _same(r, {n: got[n].cpu().numpy() for n in ("disp", "depth", "flags")}, f"frame {(s, k)}")
    ctx.close()

    # and the oracle's, on one 720p frame
    from oracle import oracle as orc
    s = [i for i, st_ in enumerate(trace.streams) if st_.width == 1280][0]
    fr = trace.streams[s].frames[0]
    ref = orc.match_frame(fr.left, fr.right, trace.streams[s].boxes[0], fr.f_px, fr.baseline_m,
                          orc.Params(**trace.params))
    compare_box_outputs(alone[(s, 0)], ref, "served 720p frame vs oracle")


def test_serving_admission_waits_for_arena(torch_cuda, trace):
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    s4k = [i for i, st_ in enumerate(trace.streams) if st_.width == 3840][0]
    budget = 2 * 3840 * 2160 + 4096          # one 4K frame's images at a time
    srv = B.Server(trace.params, lanes=2, frames_per_batch=4, image_budget_bytes=budget)
    alone = _alone(srv, trace, pinned)
    order = []
    for rep in range(3):
        for s in range(len(trace.streams)):
            for k in range(2):
                fr = trace.streams[s].frames[k]
                t = srv.submit(*pinned[s][k], trace.streams[s].boxes[k], fr.f_px, fr.baseline_m)
                order.append((t, (s, k)))
    done = {r["tag"]: r for r in srv.wait_all()}
    for t, key in order:
        assert done[t]["status"] == 0
        _same(done[t], alone[key], f"frame {key} under a small arena")
    # admitted in arrival order
    admits = [done[t]["t_admit_ns"] for t, _ in order]
    assert admits == sorted(admits)
    st = srv.stats()
    assert st["arena_peak_bytes"] <= budget
    # while a 4K frame holds the arena nothing else can be admitted beside it
    for t, (s, _) in order:
        if s != s4k:
            continue
        r = done[t]
        for t2, _ in order:
            assert t2 == t or not (r["t_admit_ns"] < done[t2]["t_admit_ns"] < r["t_done_ns"]), \
                "a frame was admitted beside a 4K frame"
    srv.close()


def test_serving_queue_full_and_too_big(torch_cuda, trace):
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    s4k = [i for i, st_ in enumerate(trace.streams) if st_.width == 3840][0]
    srv = B.Server(trace.params, lanes=1, frames_per_batch=1, max_queue=1, max_width=3840,
                   max_height=2160, image_budget_bytes=2 * 3840 * 2160 + 4096)
    fr = trace.streams[s4k].frames[0]
    tags = [srv.submit(*pinned[s4k][0], trace.streams[s4k].boxes[0], fr.f_px, fr.baseline_m)
            for _ in range(12)]
    refused = sum(t is None for t in tags)
    assert refused >= 1
    res = srv.wait_all()
    assert len(res) == 12 - refused and all(r["status"] == 0 for r in res)
    assert srv.stats()["rejected"] == refused
    big = np.zeros((2200, 3900), np.uint8)
    with pytest.raises(B.CtmError, match="fixed limit"):
        srv.submit(big, big, np.zeros((0, 5), np.int32), 1.0, 1.0)
    srv.close()


def test_serving_plain_mode_same_outputs(torch_cuda, trace):
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    a = B.Server(trace.params, lanes=2, frames_per_batch=4)
    alone = _alone(a, trace, pinned)
    a.close()
    p = B.Server(trace.params, lanes=1, frames_per_batch=1, plain=1)
    plain = _alone(p, trace, pinned)
    p.close()
    for key in alone:
        _same(plain[key], alone[key], f"plain frame {key}")


@pytest.mark.parametrize("plain", [0, 1])
def test_serving_frames_without_boxes(torch_cuda, trace, plain):
    """Frames with no boxes, or only boxes outside the image, complete with status 0
    beside ordinary frames, alone and in a mix, and leave the others' outputs unchanged."""
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    lanes, fpb = (1, 1) if plain else (2, 4)
    srv = B.Server(trace.params, lanes=lanes, frames_per_batch=fpb, plain=plain)
    alone = _alone(srv, trace, pinned)
    s0 = [i for i, st_ in enumerate(trace.streams) if st_.width == 1280][0]
    fr0 = trace.streams[s0].frames[0]
    L0, R0 = pinned[s0][0]
    outside = np.array([[2000, 10, 2100, 90, 0], [-50, -50, -1, 20, 0]], np.int32)
    t_empty = srv.submit(L0, R0, np.zeros((0, 5), np.int32), fr0.f_px, fr0.baseline_m)
    (res,) = srv.wait_all()
    assert res["tag"] == t_empty and res["status"] == 0 and res["n_boxes"] == 0
    tags = {}
    for rep in range(2):
        for s in range(len(trace.streams)):
            fr = trace.streams[s].frames[rep]
            tags[srv.submit(*pinned[s][rep], trace.streams[s].boxes[rep], fr.f_px, fr.baseline_m)] = (s, rep)
            tags[srv.submit(L0, R0, np.zeros((0, 5), np.int32), fr0.f_px, fr0.baseline_m)] = "none"
        tags[srv.submit(L0, R0, outside, fr0.f_px, fr0.baseline_m)] = "outside"
    done = srv.wait_all()
    assert len(done) == len(tags)
    for r in done:
        assert r["status"] == 0
        key = tags[r["tag"]]
        if key == "none":
            assert r["n_boxes"] == 0
        elif key == "outside":
            assert r["n_boxes"] == 2 and np.all(r["flags"] & 32) and np.all(np.isnan(r["disp"]))
        else:
            _same(r, alone[key], f"frame {key} beside frames without boxes")
    srv.close()


def test_serving_mapped_same_outputs(torch_cuda, trace):
    """A mapped server reads a gatherable frame's image bytes in place (only those
    its census needs): outputs equal the uploading server's bit for bit, for pinned
    and pageable images, alone and in a mix with frames it cannot gather (views
    8 bytes off a 16-byte boundary), which it uploads whole.  A plain server
    uploads whatever mapped says."""
    from paper_2604_07980_gb300 import binding as B
    pinned = _pinned(torch_cuda, trace)
    a = B.Server(trace.params, lanes=2, frames_per_batch=4, mapped=0)
    alone = _alone(a, trace, pinned)
    a.close()
    m = B.Server(trace.params, lanes=2, frames_per_batch=4, mapped=1)
    mapped = _alone(m, trace, pinned)
    for key in alone:
        _same(mapped[key], alone[key], f"mapped frame {key}, pinned")

    def off8(img):
        buf = np.empty(img.size + 32, np.uint8)
        o = (16 - buf.ctypes.data % 16) % 16 + 8
        view = buf[o:o + img.size].reshape(img.shape)
        view[...] = img
        return view

    tags = {}
    for s, st_ in enumerate(trace.streams):
        for k, fr in enumerate(st_.frames):
            tags[m.submit(np.ascontiguousarray(fr.left), np.ascontiguousarray(fr.right), st_.boxes[k], fr.f_px,
                          fr.baseline_m)] = (s, k)
            tags[m.submit(off8(fr.left), off8(fr.right), st_.boxes[k], fr.f_px, fr.baseline_m)] = (s, k)
    done = m.wait_all()
    assert len(done) == len(tags)
    for r in done:
        assert r["status"] == 0
        _same(r, alone[tags[r["tag"]]], f"mapped frame {tags[r['tag']]} in the mix")
    m.close()
    p = B.Server(trace.params, lanes=1, frames_per_batch=1, plain=1, mapped=1)  # plain servers upload
    assert p.config.mapped == 1
    key = next(iter(alone))
    s, k = key
    fr = trace.streams[s].frames[k]
    p.submit(*pinned[s][k], trace.streams[s].boxes[k], fr.f_px, fr.baseline_m)
    (res,) = p.wait_all()
    _same(res, alone[key], "plain server asked for mapped")
    p.close()
