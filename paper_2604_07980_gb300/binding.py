"""Thin Python binding of libctm.so (include/ctm.h).

Argument marshalling only: every step of the matching path runs in the CUDA
library.  PyTorch supplies device memory and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  There is no CPU fallback: if the
library cannot be loaded, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctm.so")

CTM_OK, CTM_EINVAL, CTM_ENOMEM, CTM_ECUDA, CTM_ENODEV, CTM_ETOOBIG, CTM_EAGAIN, CTM_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7

BOX_VALID, BOX_FB_REJECT, BOX_FEW_POINTS, BOX_NO_SEGMENT = 0x01, 0x02, 0x04, 0x08
BOX_NONPOS_DISP, BOX_EMPTY, BOX_SUBPIX_CLAMPED, BOX_FAR = 0x10, 0x20, 0x40, 0x80
BLK_VALID, BLK_FB_REJECT, BLK_FEW_POINTS, BLK_SUBPIX_CLAMPED, BLK_PRESENT = 1, 2, 4, 8, 16

# every symbol include/ctm.h declares
EXPORTS = ("ctm_status_str", "ctm_default_params", "ctm_create", "ctm_destroy",
           "ctm_census_build", "ctm_match_boxes", "ctm_match_boxes_plain", "ctm_match_batch",
           "ctm_match_batch_profiled", "ctm_match_batch_host", "ctm_match_batch_mapped", "ctm_match_boxes_noalloc",
           "ctm_noalloc_get_stats",
           "ctm_get_stats", "ctm_probe_int_rate", "ctm_probe_bounded_wait", "ctm_inject_wait_expiry", "ctm_inject_alloc_failures",
           "ctm_get_tuning",
           "ctm_set_tuning", "ctm_autotune",
           "ctm_box_points", "ctm_auto_rect", "ctm_rect_filter",
           "ctm_server_default_config", "ctm_server_create", "ctm_server_submit", "ctm_server_poll",
           "ctm_server_outstanding", "ctm_server_get_stats", "ctm_server_destroy", "ctm_server_now_ns")


class CtmError(RuntimeError):
    pass


class ctm_params(ctypes.Structure):
    _fields_ = [("win_w", ctypes.c_int32), ("win_h", ctypes.c_int32), ("sentinel", ctypes.c_int32),
                ("far_side_px", ctypes.c_int32), ("close_factor", ctypes.c_int32),
                ("far_dmin", ctypes.c_int32), ("far_dmax", ctypes.c_int32),
                ("close_dmin", ctypes.c_int32), ("close_dmax", ctypes.c_int32),
                ("dy_min", ctypes.c_int32), ("dy_max", ctypes.c_int32), ("grid_g", ctypes.c_int32),
                ("pts_side", ctypes.c_int32), ("min_pts", ctypes.c_int32), ("fb_tol", ctypes.c_int32),
                ("agg_tau_d", ctypes.c_float), ("agg_nmin", ctypes.c_int32),
                ("agg_mode", ctypes.c_int32), ("trim_frac", ctypes.c_float),
                ("max_occluders", ctypes.c_int32), ("frontal_crop", ctypes.c_float)]


class ctm_frame(ctypes.Structure):
    _fields_ = [("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pitch", ctypes.c_int32), ("box_begin", ctypes.c_int32),
                ("box_count", ctypes.c_int32), ("f_px", ctypes.c_float), ("baseline_m", ctypes.c_float)]


# The same layout as a numpy record, so that frame tables are built without a
# Python loop over frames.
FRAME_DTYPE = np.dtype([("left", np.uint64), ("right", np.uint64), ("width", np.int32), ("height", np.int32),
                        ("pitch", np.int32), ("box_begin", np.int32), ("box_count", np.int32),
                        ("f_px", np.float32), ("baseline_m", np.float32)], align=True)
assert FRAME_DTYPE.itemsize == ctypes.sizeof(ctm_frame)


class ctm_debug(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_void_p), ("cost_f", ctypes.c_void_p), ("cost_b", ctypes.c_void_p)]


class ctm_stats(ctypes.Structure):
    _fields_ = [("cost_evals", ctypes.c_uint64), ("n_blocks", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("error", ctypes.c_int32), ("census_tiles", ctypes.c_int32), ("host_bytes", ctypes.c_uint64)]


class ctm_geometry(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_float * 16), ("T", ctypes.c_float * 12), ("disp_var", ctypes.c_float),
                ("f_px", ctypes.c_float), ("baseline_m", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ctm_tuning(ctypes.Structure):
    _fields_ = [("match_threads", ctypes.c_int32), ("strip_cols", ctypes.c_int32),
                ("census_mode", ctypes.c_int32), ("queue_rounds", ctypes.c_int32),
                ("match_mode", ctypes.c_int32), ("split_ways", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class ctm_server_config(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("frames_per_batch", ctypes.c_int32),
                ("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32),
                ("max_boxes_per_frame", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("image_budget_bytes", ctypes.c_int64), ("plain", ctypes.c_int32),
                ("mapped", ctypes.c_int32)]


class ctm_request(ctypes.Structure):
    _fields_ = [("left_host", ctypes.c_void_p), ("right_host", ctypes.c_void_p),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("n_boxes", ctypes.c_int32), ("boxes_host", ctypes.c_void_p),
                ("f_px", ctypes.c_float), ("baseline_m", ctypes.c_float),
                ("disp_host", ctypes.c_void_p), ("depth_host", ctypes.c_void_p),
                ("flags_host", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class ctm_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64),
                ("lane", ctypes.c_int32), ("batch_frames", ctypes.c_int32)]


class ctm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_frames", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("arena_peak_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("max_admitted", ctypes.c_int32), ("max_lanes_busy", ctypes.c_int32)]


BLOCK_DTYPE = np.dtype([("n_pts", "<i4"), ("n_valid", "<i4"), ("d_f", "<i4"), ("dy_f", "<i4"),
                        ("d_b", "<i4"), ("dy_b", "<i4"), ("s_m", "<i4"), ("s_0", "<i4"),
                        ("s_p", "<i4"), ("d_sub", "<f4"), ("d_full", "<f4"), ("flags", "<i4")])
BLOCK_BYTES = 48
FRAME_BYTES = ctypes.sizeof(ctm_frame)

_lib = None


def lib():
    """Load libctm.so (raises if it is missing or cannot be loaded)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise CtmError(f"libctm.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    L.ctm_status_str.argtypes = [i32]
    L.ctm_status_str.restype = ctypes.c_char_p
    L.ctm_default_params.argtypes = [ctypes.POINTER(ctm_params)]
    L.ctm_default_params.restype = i32
    L.ctm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctm_params), i32, i32, i32, i32]
    L.ctm_create.restype = i32
    L.ctm_destroy.argtypes = [vp]
    L.ctm_destroy.restype = None
    L.ctm_census_build.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, vp, ctypes.c_int64, vp]
    L.ctm_census_build.restype = i32
    L.ctm_match_boxes.argtypes = [vp, vp, vp, i32, i32, i32, vp, i32, f32, f32, vp, vp, vp,
                                  ctypes.POINTER(ctm_debug), vp]
    L.ctm_match_boxes.restype = i32
    L.ctm_match_boxes_plain.argtypes = [vp, vp, vp, i32, i32, i32, vp, i32, f32, f32, vp, vp, vp, vp]
    L.ctm_match_boxes_plain.restype = i32
    L.ctm_match_batch.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(ctm_debug), i32, vp]
    L.ctm_match_batch.restype = i32
    L.ctm_match_batch_profiled.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp), vp]
    L.ctm_match_batch_profiled.restype = i32
    L.ctm_match_batch_host.argtypes = [vp, ctypes.POINTER(ctm_frame), i32, vp, i32, vp, vp, vp, vp]
    L.ctm_match_batch_host.restype = i32
    L.ctm_match_batch_mapped.argtypes = [vp, ctypes.POINTER(ctm_frame), i32, vp, i32, vp, vp, vp, vp]
    L.ctm_match_batch_mapped.restype = i32
    L.ctm_match_boxes_noalloc.argtypes = [ctypes.POINTER(ctm_params), vp, vp, i32, i32, i32, vp, i32,
                                          f32, f32, vp, vp, vp, vp]
    L.ctm_match_boxes_noalloc.restype = i32
    L.ctm_get_stats.argtypes = [vp, ctypes.POINTER(ctm_stats), vp]
    L.ctm_get_stats.restype = i32
    L.ctm_noalloc_get_stats.argtypes = [ctypes.POINTER(ctm_stats), vp]
    L.ctm_noalloc_get_stats.restype = i32
    L.ctm_probe_int_rate.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double)]
    L.ctm_probe_int_rate.restype = i32
    L.ctm_probe_bounded_wait.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    L.ctm_probe_bounded_wait.restype = i32
    L.ctm_inject_wait_expiry.argtypes = [vp]
    L.ctm_inject_wait_expiry.restype = i32
    L.ctm_inject_alloc_failures.argtypes = [i32, i32]
    L.ctm_inject_alloc_failures.restype = i32
    L.ctm_auto_rect.argtypes = [ctypes.POINTER(ctm_params), vp, vp] + [i32] * 13 + [vp, vp, vp, vp]
    L.ctm_auto_rect.restype = i32
    L.ctm_rect_filter.argtypes = [vp, i32, i32, i32]
    L.ctm_rect_filter.restype = i32
    L.ctm_box_points.argtypes = [vp, vp, vp, i32, vp, i32, vp, vp]
    L.ctm_box_points.restype = i32
    L.ctm_get_tuning.argtypes = [vp, ctypes.POINTER(ctm_tuning)]
    L.ctm_get_tuning.restype = i32
    L.ctm_set_tuning.argtypes = [vp, ctypes.POINTER(ctm_tuning)]
    L.ctm_set_tuning.restype = i32
    L.ctm_autotune.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, ctypes.POINTER(ctm_tuning),
                               ctypes.POINTER(ctypes.c_float), vp]
    L.ctm_autotune.restype = i32
    i64 = ctypes.c_int64
    L.ctm_server_default_config.argtypes = [ctypes.POINTER(ctm_server_config)]
    L.ctm_server_default_config.restype = i32
    L.ctm_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctm_params),
                                    ctypes.POINTER(ctm_server_config)]
    L.ctm_server_create.restype = i32
    L.ctm_server_submit.argtypes = [vp, ctypes.POINTER(ctm_request)]
    L.ctm_server_submit.restype = i32
    L.ctm_server_poll.argtypes = [vp, ctypes.POINTER(ctm_completion), ctypes.c_int32, i64,
                                  ctypes.POINTER(ctypes.c_int32)]
    L.ctm_server_poll.restype = i32
    L.ctm_server_outstanding.argtypes = [vp]
    L.ctm_server_outstanding.restype = i64
    L.ctm_server_get_stats.argtypes = [vp, ctypes.POINTER(ctm_server_stats)]
    L.ctm_server_get_stats.restype = i32
    L.ctm_server_destroy.argtypes = [vp]
    L.ctm_server_destroy.restype = i32
    L.ctm_server_now_ns.argtypes = []
    L.ctm_server_now_ns.restype = i64
    _lib = L
    return L


def _check(status: int, what: str):
    if status != CTM_OK:
        msg = lib().ctm_status_str(status).decode()
        err = CtmError(f"{what}: {msg} ({status})")
        err.status = status
        raise err


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise CtmError("no CUDA device: the census template matcher runs only on the GPU")
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(d: dict | None = None) -> ctm_params:
    p = ctm_params()
    _check(lib().ctm_default_params(ctypes.byref(p)), "ctm_default_params")
    for k, v in (d or {}).items():
        setattr(p, k, v)
    return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def census_build(img, factor: int = 1, win_w: int = 9, win_h: int = 7, sentinel: int = 1,
                 stream=None):
    """Census codes (uint64 stored in an int64 tensor) of a uint8 device image."""
    torch = _torch()
    assert img.dtype == torch.uint8 and img.is_cuda and img.dim() == 2
    H, W = img.shape
    pitch = img.stride(0)
    Hs, Ws = -(-H // factor), -(-W // factor)
    out = torch.empty((Hs, Ws), dtype=torch.int64, device=img.device)
    _check(lib().ctm_census_build(_ptr(img), W, H, pitch, factor, win_w, win_h, sentinel,
                                  _ptr(out), Ws, _stream(stream)), "ctm_census_build")
    return out


@dataclass
class DebugOut:
    blocks: object   # torch uint8 [n, slots, 48] (view with BLOCK_DTYPE after .cpu())
    cost_f: object   # torch int32 [n, slots, nc]
    cost_b: object

    def blocks_np(self):
        return self.blocks.cpu().numpy().reshape(-1).view(BLOCK_DTYPE).reshape(self.blocks.shape[:2])


def n_candidates(p: ctm_params) -> int:
    nd = max(p.far_dmax - p.far_dmin + 1, p.close_dmax - p.close_dmin + 1)
    return nd * (p.dy_max - p.dy_min + 1)


class Context:
    """A matching context (ctm_create) on the current CUDA device."""

    def __init__(self, params: dict | None, max_frames: int, max_width: int, max_height: int,
                 max_boxes: int):
        _torch()
        self.params = make_params(params)
        h = ctypes.c_void_p()
        _check(lib().ctm_create(ctypes.byref(h), ctypes.byref(self.params), max_frames, max_width,
                                max_height, max_boxes), "ctm_create")
        self._h = h
        self.max_frames, self.max_width, self.max_height = max_frames, max_width, max_height
        self.max_boxes = max_boxes

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ctm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def slots(self) -> int:
        return max(1, self.params.grid_g * self.params.grid_g)

    def _debug(self, n, device):
        torch = _torch()
        nc = n_candidates(self.params)
        d = DebugOut(torch.zeros((n, self.slots, BLOCK_BYTES), dtype=torch.uint8, device=device),
                     torch.zeros((n, self.slots, nc), dtype=torch.int32, device=device),
                     torch.zeros((n, self.slots, nc), dtype=torch.int32, device=device))
        c = ctm_debug(d.blocks.data_ptr(), d.cost_f.data_ptr(), d.cost_b.data_ptr())
        return d, c

    def _outputs(self, n, device):
        torch = _torch()
        return (torch.empty(n, dtype=torch.float32, device=device),
                torch.empty(n, dtype=torch.float32, device=device),
                torch.empty(n, dtype=torch.uint8, device=device))

    def match_boxes(self, left, right, boxes, f_px: float, baseline_m: float, debug: bool = False,
                    stream=None, out=None):
        """One frame.  left/right: uint8 [H, W] device tensors; boxes: int32 [n, 5] device."""
        torch = _torch()
        H, W = left.shape
        n = int(boxes.shape[0]) if boxes is not None else 0
        disp, depth, flags = out if out is not None else self._outputs(max(n, 1), left.device)
        dbg = cdbg = None
        if debug:
            dbg, cdbg = self._debug(max(n, 1), left.device)
        _check(lib().ctm_match_boxes(self._h, _ptr(left), _ptr(right), W, H, left.stride(0),
                                     _ptr(boxes), n, f_px, baseline_m, _ptr(disp), _ptr(depth),
                                     _ptr(flags), ctypes.byref(cdbg) if cdbg else None,
                                     _stream(stream)), "ctm_match_boxes")
        res = {"disp": disp[:n], "depth": depth[:n], "flags": flags[:n]}
        if debug:
            res["debug"] = dbg
        return res

    def match_boxes_plain(self, left, right, boxes, f_px: float, baseline_m: float, stream=None,
                          out=None):
        H, W = left.shape
        n = int(boxes.shape[0]) if boxes is not None else 0
        disp, depth, flags = out if out is not None else self._outputs(max(n, 1), left.device)
        _check(lib().ctm_match_boxes_plain(self._h, _ptr(left), _ptr(right), W, H, left.stride(0),
                                           _ptr(boxes), n, f_px, baseline_m, _ptr(disp),
                                           _ptr(depth), _ptr(flags), _stream(stream)),
               "ctm_match_boxes_plain")
        return {"disp": disp[:n], "depth": depth[:n], "flags": flags[:n]}

    def match_batch(self, batch: "DeviceBatch", use_graph: bool = True, debug: bool = False,
                    stream=None):
        dbg = cdbg = None
        if debug:
            dbg, cdbg = self._debug(max(batch.n_boxes, 1), batch.boxes.device)
        _check(lib().ctm_match_batch(self._h, _ptr(batch.frames), _ptr(batch.counts),
                                     _ptr(batch.boxes), _ptr(batch.disp), _ptr(batch.depth),
                                     _ptr(batch.flags), ctypes.byref(cdbg) if cdbg else None,
                                     1 if use_graph else 0, _stream(stream)), "ctm_match_batch")
        res = {"disp": batch.disp[:batch.n_boxes], "depth": batch.depth[:batch.n_boxes],
               "flags": batch.flags[:batch.n_boxes]}
        if debug:
            res["debug"] = dbg
        return res

    def match_batch_profiled(self, batch: "DeviceBatch", events, stream=None):
        """Non-graph batch recording 8 torch.cuda.Event(enable_timing=True) around its launches
        (before plan, sample+mark, census, match, aggregate; after aggregate, three times)."""
        assert len(events) == 8
        for e in events:  # torch creates the CUDA event on its first record
            if not e.cuda_event:
                e.record()
        arr = (ctypes.c_void_p * 8)(*[e.cuda_event for e in events])
        _check(lib().ctm_match_batch_profiled(self._h, _ptr(batch.frames), _ptr(batch.counts),
                                              _ptr(batch.boxes), _ptr(batch.disp), _ptr(batch.depth),
                                              _ptr(batch.flags), arr, _stream(stream)),
               "ctm_match_batch_profiled")

    def match_batch_host(self, frames_np, boxes_np, f_px, baseline_m, out=None, stream=None,
                         mapped=False):
        """Host arrays in, host arrays out (page-locked numpy views are fastest).
        frames_np: list of (left, right) uint8 [H, W] arrays; boxes_np int32 [n, 5]
        grouped by frame (column 4 = frame index).  mapped: ctm_match_batch_mapped
        (the device reads only the image bytes the census needs)."""
        nf = len(frames_np)
        tbl = np.zeros(nf, FRAME_DTYPE)
        tbl["left"] = [L.__array_interface__["data"][0] for L, _ in frames_np]
        tbl["right"] = [R.__array_interface__["data"][0] for _, R in frames_np]
        tbl["width"] = [L.shape[1] for L, _ in frames_np]
        tbl["height"] = [L.shape[0] for L, _ in frames_np]
        tbl["pitch"] = [L.strides[0] for L, _ in frames_np]
        return self._host_call(tbl, boxes_np, f_px, baseline_m, out, stream, mapped)

    def match_batch_host_packed(self, images, boxes_np, f_px, baseline_m, out=None, stream=None,
                                mapped=False):
        """Like match_batch_host for frames packed in one host array images[F, 2, H, W]
        (left, right; a frame-grabber ring buffer): the frame table is computed from
        the array's strides, and frames stored back to back go in one copy per sub-batch."""
        if images.ndim != 4 or images.shape[1] != 2 or images.dtype != np.uint8 or images.strides[3] != 1:
            raise ValueError("images must be uint8 [F, 2, H, W] with unit column stride")
        nf, _, H, W = images.shape
        base = images.__array_interface__["data"][0]
        tbl = np.zeros(nf, FRAME_DTYPE)
        tbl["left"] = base + np.arange(nf, dtype=np.uint64) * np.uint64(images.strides[0])
        tbl["right"] = tbl["left"] + np.uint64(images.strides[1])
        tbl["width"] = W
        tbl["height"] = H
        tbl["pitch"] = images.strides[2]
        return self._host_call(tbl, boxes_np, f_px, baseline_m, out, stream, mapped)

    def _host_call(self, tbl, boxes_np, f_px, baseline_m, out, stream, mapped=False):
        nf = len(tbl)
        n = int(boxes_np.shape[0])
        counts = np.bincount(boxes_np[:, 4], minlength=nf) if n else np.zeros(nf, np.int64)
        tbl["box_count"] = counts[:nf]
        tbl["box_begin"][1:] = np.cumsum(counts[:nf])[:-1]
        tbl["f_px"] = f_px
        tbl["baseline_m"] = baseline_m
        if out is None:
            out = (np.empty(max(n, 1), np.float32), np.empty(max(n, 1), np.float32),
                   np.empty(max(n, 1), np.uint8))
        disp, depth, flags = out
        bx = np.ascontiguousarray(boxes_np, dtype=np.int32)
        fn = lib().ctm_match_batch_mapped if mapped else lib().ctm_match_batch_host
        _check(fn(self._h, tbl.ctypes.data_as(ctypes.POINTER(ctm_frame)), nf, bx.ctypes.data, n,
                  disp.ctypes.data, depth.ctypes.data, flags.ctypes.data, _stream(stream)),
               "ctm_match_batch_mapped" if mapped else "ctm_match_batch_host")
        return {"disp": disp[:n], "depth": depth[:n], "flags": flags[:n]}

    def get_tuning(self) -> dict:
        t = ctm_tuning()
        _check(lib().ctm_get_tuning(self._h, ctypes.byref(t)), "ctm_get_tuning")
        return t.as_dict()

    def set_tuning(self, **fields):
        t = ctm_tuning(**{**self.get_tuning(), **fields})
        _check(lib().ctm_set_tuning(self._h, ctypes.byref(t)), "ctm_set_tuning")

    def autotune(self, batch: "DeviceBatch", reps: int = 3, stream=None) -> tuple[dict, float]:
        """Time candidate launch shapes on this batch, keep the fastest; returns it and ms per call."""
        t = ctm_tuning()
        ms = ctypes.c_float(0.0)
        _check(lib().ctm_autotune(self._h, _ptr(batch.frames), _ptr(batch.counts), _ptr(batch.boxes),
                                  _ptr(batch.disp), _ptr(batch.depth), _ptr(batch.flags), int(reps),
                                  ctypes.byref(t), ctypes.byref(ms), _stream(stream)), "ctm_autotune")
        return t.as_dict(), float(ms.value)

    def inject_wait_expiry(self):
        """Arm the test-only fault injection (ctm_inject_wait_expiry) for the next direct call."""
        _check(lib().ctm_inject_wait_expiry(self._h), "ctm_inject_wait_expiry")

    def stats(self, stream=None) -> dict:
        s = ctm_stats()
        _check(lib().ctm_get_stats(self._h, ctypes.byref(s), _stream(stream)), "ctm_get_stats")
        return {"cost_evals": int(s.cost_evals), "n_blocks": int(s.n_blocks), "n_boxes": int(s.n_boxes),
                "error": int(s.error), "census_tiles": int(s.census_tiles), "host_bytes": int(s.host_bytes)}


class DeviceBatch:
    """Device-resident batch: frame descriptors, counts, boxes and outputs.

    frames: list of (left, right) uint8 device tensors; boxes: int32 [n, 5] with the
    frame index in column 4, grouped by frame; calib: list of (f_px, baseline_m)."""

    def __init__(self, frames, boxes, calib, device=None):
        torch = _torch()
        device = device or frames[0][0].device
        n = int(boxes.shape[0])
        bnp = boxes.cpu().numpy() if hasattr(boxes, "cpu") else np.asarray(boxes)
        counts = np.bincount(bnp[:, 4], minlength=len(frames)) if n else np.zeros(len(frames), int)
        begins = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
        arr = (ctm_frame * len(frames))()
        for i, (L, R) in enumerate(frames):
            arr[i] = ctm_frame(L.data_ptr(), R.data_ptr(), L.shape[1], L.shape[0], L.stride(0),
                               int(begins[i]), int(counts[i]), float(calib[i][0]), float(calib[i][1]))
        raw = np.frombuffer(bytes(arr), dtype=np.uint8)
        self.frames_keep = frames
        self.frames = torch.from_numpy(raw.copy()).to(device)
        self.counts = torch.tensor([len(frames), n], dtype=torch.int32, device=device)
        self.boxes = torch.as_tensor(np.ascontiguousarray(bnp, dtype=np.int32), device=device)
        self.n_boxes = n
        self.n_frames = len(frames)
        self.disp = torch.empty(max(n, 1), dtype=torch.float32, device=device)
        self.depth = torch.empty(max(n, 1), dtype=torch.float32, device=device)
        self.flags = torch.empty(max(n, 1), dtype=torch.uint8, device=device)


def geometries_to_device(geometries, device="cuda"):
    """ctm_geometry array in device memory from dicts with Q (4x4), T (3x4), disp_var,
    f_px, baseline_m, width, height."""
    torch = _torch()
    arr = (ctm_geometry * max(len(geometries), 1))()
    for i, g in enumerate(geometries):
        arr[i].Q[:] = [float(x) for x in np.asarray(g["Q"], np.float64).ravel()]
        arr[i].T[:] = [float(x) for x in np.asarray(g["T"], np.float64).ravel()]
        arr[i].disp_var = float(g["disp_var"])
        arr[i].f_px = float(g["f_px"])
        arr[i].baseline_m = float(g["baseline_m"])
        arr[i].width = int(g["width"])
        arr[i].height = int(g["height"])
    raw = np.frombuffer(bytes(arr), dtype=np.uint8)
    return torch.from_numpy(raw.copy()).to(device), len(geometries)


def box_points(boxes, disp, flags, geo, n_geo: int, out=None, stream=None):
    """Sec. 4.3.6 per box on the device: float32 [n, 8] (camera x y z, vehicle x y z,
    sigma_Z^2, W).  boxes int32 [n, 5] (column 4 = frame index into geo), disp float32 [n],
    flags uint8 [n], geo from geometries_to_device."""
    torch = _torch()
    n = int(boxes.shape[0])
    if out is None:
        out = torch.empty((max(n, 1), 8), dtype=torch.float32, device=boxes.device)
    _check(lib().ctm_box_points(_ptr(boxes), _ptr(disp), _ptr(flags), n, _ptr(geo), int(n_geo), _ptr(out),
                                _stream(stream)), "ctm_box_points")
    return out[:n]


def auto_rect(left, right, roi, dmin: int, dmax: int, delta_min: int, delta_max: int, d_thresh: int,
              fb_tol: int = 1, params: dict | None = None, stream=None):
    """Sec. 5.1 offset search on the device (census matching): returns (delta*, counts) as
    device tensors; left/right uint8 [H, W] device tensors, roi = (x0, y0, x1, y1)."""
    torch = _torch()
    p = make_params(params)
    H, W = left.shape
    census = torch.empty((2, H, W), dtype=torch.int64, device=left.device)
    counts = torch.empty(delta_max - delta_min + 1, dtype=torch.int64, device=left.device)
    delta = torch.empty(1, dtype=torch.int32, device=left.device)
    _check(lib().ctm_auto_rect(ctypes.byref(p), _ptr(left), _ptr(right), W, H, left.stride(0), roi[0], roi[1],
                               roi[2], roi[3], dmin, dmax, delta_min, delta_max, d_thresh, fb_tol, _ptr(census),
                               _ptr(counts), _ptr(delta), _stream(stream)), "ctm_auto_rect")
    return delta, counts


def rect_filter(estimates, prev: int, max_step: int) -> int:
    v = np.ascontiguousarray(estimates, dtype=np.int32)
    return int(lib().ctm_rect_filter(v.ctypes.data if len(v) else None, len(v), prev, max_step))


def _host_ptr(a):
    """Address and row pitch of a 2-D uint8 host array (numpy or CPU torch tensor)."""
    if hasattr(a, "data_ptr"):
        assert a.dtype.itemsize == 1 and not a.is_cuda and a.dim() == 2 and a.stride(1) == 1
        return a.data_ptr(), a.stride(0), a.shape[0], a.shape[1]
    assert a.dtype == np.uint8 and a.ndim == 2 and a.strides[1] == 1
    return a.ctypes.data, a.strides[0], a.shape[0], a.shape[1]


class Server:
    """The serving loop (ctm_server_*) on the current CUDA device.

    submit() queues one frame (host images, host boxes) and returns its tag;
    poll() returns finished frames with their outputs and timestamps.  The
    arrays passed to submit() are kept alive here until their frame completes;
    page-locked images (pinned torch tensors) let the uploads run async."""

    def __init__(self, params: dict | None = None, **config):
        _torch()
        self.params = make_params(params)
        cfg = ctm_server_config()
        _check(lib().ctm_server_default_config(ctypes.byref(cfg)), "ctm_server_default_config")
        for k, v in config.items():
            setattr(cfg, k, v)
        self.config = cfg
        h = ctypes.c_void_p()
        _check(lib().ctm_server_create(ctypes.byref(h), ctypes.byref(self.params), ctypes.byref(cfg)),
               "ctm_server_create")
        self._h = h
        self._live = {}
        self._next_tag = 1

    def submit(self, left, right, boxes, f_px: float, baseline_m: float, tag: int | None = None):
        """Queue a frame; returns its tag, or None when the admission queue is full."""
        lp, pitch, H, W = _host_ptr(left)
        rp, rpitch, H2, W2 = _host_ptr(right)
        assert (H, W) == (H2, W2) and rpitch == pitch
        bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 5)
                                  if np.asarray(boxes).size else np.zeros((0, 5), np.int32))
        n = int(bx.shape[0])
        out = (np.empty(max(n, 1), np.float32), np.empty(max(n, 1), np.float32),
               np.empty(max(n, 1), np.uint8))
        if tag is None:
            tag = self._next_tag
            self._next_tag += 1
        req = ctm_request(lp, rp, W, H, pitch, n, bx.ctypes.data, float(f_px), float(baseline_m),
                          out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data, int(tag))
        self._live[int(tag)] = (left, right, bx, out)
        st = lib().ctm_server_submit(self._h, ctypes.byref(req))
        if st == CTM_EAGAIN:
            del self._live[int(tag)]
            return None
        if st != CTM_OK:
            del self._live[int(tag)]
            _check(st, "ctm_server_submit")
        return int(tag)

    def poll(self, max_n: int = 256, timeout_us: int = 0) -> list:
        """Finished frames: dicts with tag, status, disp/depth/flags, timestamps (ns), lane."""
        arr = (ctm_completion * max_n)()
        n = ctypes.c_int32(0)
        _check(lib().ctm_server_poll(self._h, arr, max_n, int(timeout_us), ctypes.byref(n)),
               "ctm_server_poll")
        res = []
        for i in range(n.value):
            c = arr[i]
            _, _, _, out = self._live.pop(int(c.tag))
            k = int(c.n_boxes)
            res.append({"tag": int(c.tag), "status": int(c.status), "n_boxes": k,
                        "disp": out[0][:k], "depth": out[1][:k], "flags": out[2][:k],
                        "t_submit_ns": int(c.t_submit_ns), "t_admit_ns": int(c.t_admit_ns),
                        "t_launch_ns": int(c.t_launch_ns), "t_done_ns": int(c.t_done_ns),
                        "lane": int(c.lane), "batch_frames": int(c.batch_frames)})
        return res

    def wait_all(self, timeout_s: float = 120.0) -> list:
        """Poll until every submitted frame has completed."""
        import time
        out = []
        t_end = time.monotonic() + timeout_s
        while self._live:
            if time.monotonic() > t_end:
                raise CtmError(f"server: {len(self._live)} frames still outstanding after {timeout_s} s")
            out += self.poll(256, 20000)
        return out

    def outstanding(self) -> int:
        return int(lib().ctm_server_outstanding(self._h))

    def stats(self) -> dict:
        s = ctm_server_stats()
        _check(lib().ctm_server_get_stats(self._h, ctypes.byref(s)), "ctm_server_get_stats")
        return {f: int(getattr(s, f)) for f, _ in ctm_server_stats._fields_}

    @staticmethod
    def now_ns() -> int:
        return int(lib().ctm_server_now_ns())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ctm_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def frames_to_device(frames, device="cuda"):
    """[(left, right)] uint8 device tensors from objects with .left/.right numpy arrays."""
    torch = _torch()
    return [(torch.from_numpy(np.ascontiguousarray(f.left)).to(device),
             torch.from_numpy(np.ascontiguousarray(f.right)).to(device)) for f in frames]


def probe_bounded_wait() -> tuple[int, float]:
    """Run the bounded-wait probe: (expired flag, kernel milliseconds)."""
    _torch()
    flag = ctypes.c_int(0)
    ms = ctypes.c_float(0.0)
    _check(lib().ctm_probe_bounded_wait(ctypes.byref(flag), ctypes.byref(ms)), "ctm_probe_bounded_wait")
    return int(flag.value), float(ms.value)


def probe_int_rate(kind: int, iters: int = 4096) -> float:
    """Operations per SM clock per SM: 32-bit popcount (kind 0), 3-input xor (1), packed fp16
    greater-than (2), 32-bit add (3), 32-bit multiply-add (4) or packed fp16 fused
    multiply-add with saturation (5)."""
    _torch()
    v = ctypes.c_double(0.0)
    _check(lib().ctm_probe_int_rate(kind, iters, ctypes.byref(v)), "ctm_probe_int_rate")
    return float(v.value)
