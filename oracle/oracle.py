"""Python view of the plain CPU oracle (oracle/ctm_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA library; only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import it.  It
never imports the library package and the library never imports it.

``build()`` compiles ``ctm_oracle.c`` with gcc (no fast-math, no FP contraction)
into ``oracle/_build/libctm_oracle.so``; the wrappers only marshal numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctm_oracle.c")
_HDR = os.path.join(_HERE, "ctm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libctm_oracle.so")

_lib = None


def compile_source(src: str, so: str) -> str:
    """gcc one oracle source file (plain C11, no fast-math, no FP contraction) into
    the shared library ``so``; the header is found beside ``_SRC``."""
    tmp = so + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-Wall", "-Wextra", "-I", _HERE, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        compile_source(_SRC, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f32p = ctypes.POINTER(ctypes.c_float)
        L.orc_census.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]
        L.orc_census.restype = None
        L.orc_subpixel.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.orc_subpixel.restype = ctypes.c_float
        L.orc_aggregate.argtypes = [f32p, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_float, f32p]
        L.orc_aggregate.restype = ctypes.c_int
        L.orc_depth.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
        L.orc_depth.restype = ctypes.c_float
        L.orc_auto_rect.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 16 + [ctypes.c_void_p]
        L.orc_auto_rect.restype = ctypes.c_int
        L.orc_rect_filter.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_rect_filter.restype = ctypes.c_int
        L.orc_box_points.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.orc_box_points.restype = None
        L.orc_match_frame.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      i32p, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_void_p, f32p, f32p, u8p, ctypes.c_void_p,
                                      i32p, i32p]
        L.orc_match_frame.restype = ctypes.c_int
        _lib = L
    return _lib


@dataclass
class Params:
    """Mirror of ``orc_params``; defaults are the 1920x1080 single-frame workload's."""
    win_w: int = 9
    win_h: int = 7
    sentinel: int = 1
    far_side_px: int = 40
    close_factor: int = 2
    far_dmin: int = 0
    far_dmax: int = 31
    close_dmin: int = 0
    close_dmax: int = 127
    dy_min: int = 0
    dy_max: int = 0
    grid_g: int = 4
    pts_side: int = 16
    min_pts: int = 16
    fb_tol: int = 1
    agg_tau_d: float = 1.0
    agg_nmin: int = 6
    agg_mode: int = 0
    trim_frac: float = 0.2
    max_occluders: int = 16
    frontal_crop: float = 0.0


class _CParams(ctypes.Structure):
    _fields_ = [(f.name, ctypes.c_float if f.type in (float, "float") else ctypes.c_int32)
                for f in fields(Params)]


def _cparams(p: Params) -> _CParams:
    return _CParams(**{f.name: getattr(p, f.name) for f in fields(Params)})


BLOCK_DTYPE = np.dtype([("n_pts", "<i4"), ("n_valid", "<i4"), ("d_f", "<i4"), ("dy_f", "<i4"),
                        ("d_b", "<i4"), ("dy_b", "<i4"), ("s_m", "<i4"), ("s_0", "<i4"),
                        ("s_p", "<i4"), ("d_sub", "<f4"), ("d_full", "<f4"), ("flags", "<i4")])

BLK_VALID, BLK_FB_REJECT, BLK_FEW_POINTS, BLK_SUBPIX_CLAMPED, BLK_PRESENT = 1, 2, 4, 8, 16
BOX_VALID, BOX_FB_REJECT, BOX_FEW_POINTS, BOX_NO_SEGMENT = 1, 2, 4, 8
BOX_NONPOS_DISP, BOX_EMPTY, BOX_SUBPIX_CLAMPED, BOX_FAR = 16, 32, 64, 128


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def census(img: np.ndarray, k: int = 1, win_w: int = 9, win_h: int = 7,
           sentinel: int = 1) -> np.ndarray:
    """Census of I(k x, k y); returns uint64 [ceil(H/k), ceil(W/k)]."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    Hs, Ws = -(-H // k), -(-W // k)
    out = np.zeros((Hs, Ws), dtype=np.uint64)
    lib().orc_census(_ptr(img, ctypes.c_uint8), W, H, W, k, win_w, win_h, sentinel,
                     _ptr(out, ctypes.c_uint64))
    return out


def subpixel(d_star: int, s_m: int, s_0: int, s_p: int) -> float:
    return float(lib().orc_subpixel(d_star, s_m, s_0, s_p))


def aggregate(vals, tau_d: float, nmin: int, mode: int = 0, trim_frac: float = 0.2):
    v = np.ascontiguousarray(vals, dtype=np.float32)
    out = ctypes.c_float(0.0)
    ok = lib().orc_aggregate(_ptr(v, ctypes.c_float), len(v), tau_d, nmin, mode, trim_frac,
                             ctypes.byref(out))
    return float(out.value) if ok else None


def depth(f_px: float, baseline_m: float, d: float) -> float:
    return float(lib().orc_depth(f_px, baseline_m, d))


def n_candidates(p: Params) -> int:
    nd = max(p.far_dmax - p.far_dmin + 1, p.close_dmax - p.close_dmin + 1)
    return nd * (p.dy_max - p.dy_min + 1)


def match_frame(L: np.ndarray, R: np.ndarray, boxes: np.ndarray, f_px: float,
                baseline_m: float, p: Params, debug: bool = False):
    """Algorithm 2 on one frame.

    boxes: int32 [n, 5] (x0, y0, x1, y1, frame) half-open full-res rectangles.
    Returns dict with disp, depth, flags and, with debug, blocks
    (structured [n, slots]) and cost_f / cost_b ([n, slots, NC]).
    """
    L = np.ascontiguousarray(L, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint8)
    H, W = L.shape
    assert R.shape == L.shape
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 5)
    n = boxes.shape[0]
    slots = p.grid_g * p.grid_g
    nc = n_candidates(p)
    disp = np.zeros(n, np.float32)
    dep = np.zeros(n, np.float32)
    flg = np.zeros(n, np.uint8)
    blk = cf = cb = None
    if debug:
        blk = np.zeros((n, slots), BLOCK_DTYPE)
        cf = np.zeros((n, slots, nc), np.int32)
        cb = np.zeros((n, slots, nc), np.int32)
    cp = _cparams(p)
    rc = lib().orc_match_frame(
        _ptr(L, ctypes.c_uint8), _ptr(R, ctypes.c_uint8), W, H, W,
        _ptr(boxes, ctypes.c_int32), n, f_px, baseline_m, ctypes.cast(ctypes.byref(cp), ctypes.c_void_p),
        _ptr(disp, ctypes.c_float), _ptr(dep, ctypes.c_float), _ptr(flg, ctypes.c_uint8),
        blk.ctypes.data if blk is not None else None,
        _ptr(cf, ctypes.c_int32) if cf is not None else None,
        _ptr(cb, ctypes.c_int32) if cb is not None else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (status {rc})")
    out = {"disp": disp, "depth": dep, "flags": flg}
    if debug:
        out.update(blocks=blk, cost_f=cf, cost_b=cb)
    return out


def match_batch(frames, boxes: np.ndarray, p: Params, debug: bool = False):
    """Frames: list of (L, R, f_px, baseline_m); boxes [n, 5] with the frame index in
    column 4, grouped by frame.  Runs match_frame per frame and concatenates."""
    boxes = np.asarray(boxes, dtype=np.int32).reshape(-1, 5)
    outs = []
    for fi, (L, R, f_px, b_m) in enumerate(frames):
        sel = boxes[:, 4] == fi
        outs.append(match_frame(L, R, boxes[sel], f_px, b_m, p, debug=debug))
    res = {key: np.concatenate([o[key] for o in outs]) for key in outs[0]} if outs else {}
    return res


class _CGeometry(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_double * 16), ("T", ctypes.c_double * 12), ("disp_var", ctypes.c_double),
                ("f_px", ctypes.c_double), ("baseline_m", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


def box_points(boxes: np.ndarray, disp: np.ndarray, flags: np.ndarray, geometries) -> np.ndarray:
    """Sec. 4.3.6 reprojection + vehicle transform + depth variance per box (float64 [n, 8]:
    camera x y z, vehicle x y z, sigma_Z^2, W).  geometries: list of dicts with Q (4x4),
    T (3x4), disp_var, f_px, baseline_m, width, height; box i uses geometries[boxes[i, 4]]."""
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 5)
    n = boxes.shape[0]
    disp = np.ascontiguousarray(disp, dtype=np.float32)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    arr = (_CGeometry * max(len(geometries), 1))()
    for i, g in enumerate(geometries):
        arr[i].Q[:] = [float(x) for x in np.asarray(g["Q"], np.float64).ravel()]
        arr[i].T[:] = [float(x) for x in np.asarray(g["T"], np.float64).ravel()]
        arr[i].disp_var = float(g["disp_var"])
        arr[i].f_px = float(g["f_px"])
        arr[i].baseline_m = float(g["baseline_m"])
        arr[i].width = int(g["width"])
        arr[i].height = int(g["height"])
    out = np.empty((max(n, 1), 8), np.float64)
    lib().orc_box_points(boxes.ctypes.data, disp.ctypes.data, flags.ctypes.data, n,
                         ctypes.addressof(arr), len(geometries), out.ctypes.data)
    return out[:n]


def auto_rect(L: np.ndarray, R: np.ndarray, roi, dmin: int, dmax: int, delta_min: int, delta_max: int,
              d_thresh: int, fb_tol: int = 1, win_w: int = 9, win_h: int = 7, sentinel: int = 1):
    """Sec. 5.1 offset search with census matching; returns (delta*, counts per delta)."""
    L = np.ascontiguousarray(L, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint8)
    H, W = L.shape
    counts = np.zeros(delta_max - delta_min + 1, np.int64)
    best = lib().orc_auto_rect(L.ctypes.data, R.ctypes.data, W, H, W, win_w, win_h, sentinel,
                               roi[0], roi[1], roi[2], roi[3], dmin, dmax, delta_min, delta_max,
                               d_thresh, fb_tol, counts.ctypes.data)
    return int(best), counts


def rect_filter(estimates, prev: int, max_step: int) -> int:
    v = np.ascontiguousarray(estimates, dtype=np.int32)
    return int(lib().orc_rect_filter(v.ctypes.data, len(v), prev, max_step))
