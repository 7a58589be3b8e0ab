"""Frame tables the host entry points build (CPU only: the library call is
replaced by a recorder).  The packed form computes every pointer from the
array's strides; both forms give each frame its box range and calibration."""
import ctypes

import numpy as np

from paper_2604_07980_gb300 import binding as B


class _Recorder:
    def __init__(self):
        self.calls = []

    def ctm_match_batch_host(self, *args):
        self.calls.append(args)
        return B.CTM_OK


def _table(monkeypatch, call):
    rec = _Recorder()
    monkeypatch.setattr(B, "lib", lambda: rec)
    monkeypatch.setattr(B, "_stream", lambda s: None)
    ctx = object.__new__(B.Context)
    ctx._h = None
    out = call(ctx)
    (h, tbl_ptr, nf, bx, n, disp, depth, flags, stream), = rec.calls
    raw = ctypes.string_at(ctypes.addressof(tbl_ptr.contents), nf * B.FRAME_DTYPE.itemsize)
    return np.frombuffer(raw, dtype=B.FRAME_DTYPE), n, out


def test_frame_dtype_matches_struct():
    assert B.FRAME_DTYPE.itemsize == ctypes.sizeof(B.ctm_frame)
    for name, _ in B.ctm_frame._fields_:
        assert B.FRAME_DTYPE.fields[name][1] == getattr(B.ctm_frame, name).offset, name


def test_packed_and_list_tables(monkeypatch):
    F, H, W = 5, 24, 40
    images = np.zeros((F, 2, H, W), np.uint8)
    boxes = np.array([[0, 0, 4, 4, f] for f in (0, 0, 1, 3, 3, 3)], np.int32)
    fpx = [1000.0 + i for i in range(F)]
    tbl, n, out = _table(monkeypatch, lambda c: c.match_batch_host_packed(images, boxes, fpx, 0.25))
    base = images.__array_interface__["data"][0]
    assert n == 6 and out["disp"].shape == (6,)
    for i in range(F):
        assert tbl["left"][i] == base + i * 2 * H * W
        assert tbl["right"][i] == base + i * 2 * H * W + H * W
    assert list(tbl["width"]) == [W] * F and list(tbl["height"]) == [H] * F and list(tbl["pitch"]) == [W] * F
    assert list(tbl["box_begin"]) == [0, 2, 3, 3, 6] and list(tbl["box_count"]) == [2, 1, 0, 3, 0]
    assert np.allclose(tbl["f_px"], fpx) and np.allclose(tbl["baseline_m"], 0.25)
    frames = [(images[i, 0], images[i, 1]) for i in range(F)]
    tbl2, _, _ = _table(monkeypatch, lambda c: c.match_batch_host(frames, boxes, fpx, [0.25] * F))
    assert tbl2.tobytes() == tbl.tobytes()


def test_packed_rejects_bad_layouts(monkeypatch):
    import pytest
    with pytest.raises(ValueError):
        _table(monkeypatch, lambda c: c.match_batch_host_packed(np.zeros((2, 3, 4, 4), np.uint8),
                                                                np.zeros((0, 5), np.int32), 1.0, 1.0))
    with pytest.raises(ValueError):
        _table(monkeypatch, lambda c: c.match_batch_host_packed(np.zeros((2, 2, 4, 4), np.uint16),
                                                                np.zeros((0, 5), np.int32), 1.0, 1.0))
