"""Seeded synthetic stereo workloads.

This module only makes inputs: textured image pairs with planted boxes at known
disparities, the boxes, and the matching parameters of each named workload.  It
holds none of the matching arithmetic, and both the CUDA library's tests and the
CPU oracle consume what it returns.

Recipe (all numpy, PCG64, seed = 1000 + workload index, per-frame sub-seeds):
  * texture: i.i.d. N(0,1) noise, separable Gaussian blur (sigma 1.5, radius 5,
    reflected border), affine map to mean 128 / std 40;
  * left image: the background texture, then every box's own texture painted in
    ascending bottom-y order (a lower bottom edge is nearer, so it is painted on
    top), rounded and clipped to uint8;
  * right image: the background at disparity 0 and each box texture shifted left
    by its float d_true using bilinear sampling, painted in the same order, then
    gain, offset and N(0, sigma) noise, rounded and clipped;
  * optional occluding strips: a vertical strip inside a box, full box height, at
    a larger disparity, emitted as its own box whose bottom edge is 1-10 px lower.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass, field

import numpy as np

F_PX = 2000.0       # focal length in px (the truck-camera example of Sec. 1.2)
BASELINE_M = 0.30   # stereo baseline in m (same example)


@dataclass
class Frame:
    left: np.ndarray      # uint8 [H, W]
    right: np.ndarray     # uint8 [H, W]
    f_px: float = F_PX
    baseline_m: float = BASELINE_M

    @property
    def shape(self):
        return self.left.shape


@dataclass
class Workload:
    name: str
    frames: list
    boxes: np.ndarray          # int32 [n, 5]: x0, y0, x1, y1, frame (grouped by frame)
    d_true: np.ndarray         # float32 [n], full-res px
    params: dict               # matching parameters (names of the C parameter block)
    meta: dict = field(default_factory=dict)

    @property
    def n_boxes(self) -> int:
        return int(self.boxes.shape[0])


# Matching parameters per workload.  Keys are the fields of the C parameter block.
PARAMS = {
    # 640x480 pair, 7x7 census, every box a 3x3 grid at full resolution.
    "pair640": dict(win_w=7, win_h=7, sentinel=1, far_side_px=0, close_factor=1,
                    far_dmin=0, far_dmax=63, close_dmin=0, close_dmax=63, dy_min=0, dy_max=0,
                    grid_g=3, pts_side=16, min_pts=16, fb_tol=1, agg_tau_d=1.0, agg_nmin=3,
                    agg_mode=0, trim_frac=0.2, max_occluders=16),
    # 1920x1080 single frame, far/close split, 9x7 census.
    "frame1080": dict(win_w=9, win_h=7, sentinel=1, far_side_px=40, close_factor=2,
                      far_dmin=0, far_dmax=31, close_dmin=0, close_dmax=127, dy_min=0, dy_max=0,
                      grid_g=4, pts_side=16, min_pts=16, fb_tol=1, agg_tau_d=1.0, agg_nmin=6,
                      agg_mode=0, trim_frac=0.2, max_occluders=16),
    # 32 x 1920x1200 batch with occluding strips.
    "batch32x1200": dict(win_w=9, win_h=7, sentinel=1, far_side_px=40, close_factor=2,
                         far_dmin=0, far_dmax=127, close_dmin=0, close_dmax=63, dy_min=0, dy_max=0,
                         grid_g=4, pts_side=16, min_pts=16, fb_tol=1, agg_tau_d=1.0, agg_nmin=6,
                         agg_mode=0, trim_frac=0.2, max_occluders=16),
    # 8 x 3840x2160 batch, 25 blocks, trimmed mean.
    "batch8x2160": dict(win_w=9, win_h=7, sentinel=1, far_side_px=40, close_factor=2,
                        far_dmin=0, far_dmax=63, close_dmin=0, close_dmax=127, dy_min=0, dy_max=0,
                        grid_g=5, pts_side=16, min_pts=16, fb_tol=1, agg_tau_d=1.0, agg_nmin=9,
                        agg_mode=1, trim_frac=0.2, max_occluders=16),
}
PARAMS["serving"] = dict(PARAMS["frame1080"])

WORKLOAD_INDEX = {"pair640": 0, "frame1080": 1, "batch32x1200": 2, "batch8x2160": 3, "serving": 4}


# --------------------------------------------------------------------------- textures

def _gauss_taps(sigma: float = 1.5, radius: int = 5) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur_axis(a: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    r = (len(taps) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    p = np.pad(a, pad, mode="reflect")
    n = a.shape[axis]
    out = np.zeros_like(a)
    for t, w in enumerate(taps):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(t, t + n)
        out += w * p[tuple(sl)]
    return out


def texture(rng: np.random.Generator, h: int, w: int, mean: float = 128.0,
            std: float = 40.0) -> np.ndarray:
    """Blurred white noise (sigma 1.5) mapped to the given mean and std (float64)."""
    taps = _gauss_taps()
    a = rng.standard_normal((max(h, 1), max(w, 1)))
    a = _blur_axis(_blur_axis(a, taps, 0), taps, 1)
    s = a.std()
    a = (a - a.mean()) / (s if s > 0 else 1.0)
    return a * std + mean


def _to_u8(a: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(a), 0, 255).astype(np.uint8)


def _paint(Lf: np.ndarray, Rf: np.ndarray, rng: np.random.Generator, box, d: float) -> None:
    """Paint one object texture: into the left image on the box, into the right
    image shifted left by d (bilinear along x)."""
    H, W = Lf.shape
    x0, y0, x1, y1 = (int(v) for v in box[:4])
    w, h = x1 - x0, y1 - y0
    if w <= 0 or h <= 0:
        return
    T = texture(rng, h, w + 2)
    ys0, ys1 = max(y0, 0), min(y1, H)
    if ys1 <= ys0:
        return
    rows = slice(ys0 - y0, ys1 - y0)
    lx0, lx1 = max(x0, 0), min(x1, W)
    if lx1 > lx0:
        Lf[ys0:ys1, lx0:lx1] = T[rows, lx0 - x0:lx1 - x0]
    # right image: pixel x' shows object coordinate u = x' - x0 + d, u in [0, w)
    xr0 = int(np.ceil(x0 - d))
    xr1 = int(np.ceil(x1 - d))
    xr0c, xr1c = max(xr0, 0), min(xr1, W)
    if xr1c > xr0c:
        u = np.arange(xr0c, xr1c, dtype=np.float64) - x0 + d
        u = np.clip(u, 0.0, w - 1e-9)
        iu = np.floor(u).astype(np.int64)
        fu = u - iu
        Tr = T[rows]
        Rf[ys0:ys1, xr0c:xr1c] = Tr[:, iu] * (1.0 - fu) + Tr[:, iu + 1] * fu


def _loguniform(rng, lo, hi):
    return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))


def _box_of_side(rng, side, W, H, aspect=(0.5, 1.5)):
    a = rng.uniform(*aspect)  # h / w
    if a >= 1.0:
        h, w = side, side / a
    else:
        w, h = side, side * a
    w = int(max(2, min(round(w), W)))
    h = int(max(2, min(round(h), H)))
    x0 = int(rng.integers(0, W - w + 1))
    y0 = int(rng.integers(0, H - h + 1))
    return [x0, y0, x0 + w, y0 + h]


def _render(rng, W, H, boxes_f, d_f, gain, offset, sigma):
    """Background at disparity 0 plus boxes painted nearest-last."""
    bg = texture(rng, H, W)
    Lf = bg.copy()
    Rf = bg.copy()
    order = sorted(range(len(boxes_f)), key=lambda i: (boxes_f[i][3], i))
    for i in order:
        _paint(Lf, Rf, rng, boxes_f[i], float(d_f[i]))
    L = _to_u8(Lf)
    R = _to_u8(gain * Rf + offset + rng.normal(0.0, sigma, size=Rf.shape))
    return L, R


# --------------------------------------------------------------------------- workloads

def _frame_rng(seed, fi):
    return np.random.Generator(np.random.PCG64([seed, fi]))


def pair640(seed: int = 1000, W: int = 640, H: int = 480, n_boxes: int = 4, side: int = 48,
            d_range=(2.0, 60.0)) -> Workload:
    """One 640x480 pair, non-overlapping 48x48 boxes, gain 1, offset +10, sigma 2."""
    rng = _frame_rng(seed, 0)
    boxes, d = [], []
    tries = 0
    while len(boxes) < n_boxes and tries < 10000:
        tries += 1
        x0 = int(rng.integers(int(d_range[1]) + 8, W - side - 8 + 1))
        y0 = int(rng.integers(8, H - side - 8 + 1))
        b = [x0, y0, x0 + side, y0 + side]
        if any(not (b[2] <= o[0] or o[2] <= b[0] or b[3] <= o[1] or o[3] <= b[1]) for o in boxes):
            continue
        boxes.append(b)
        d.append(rng.uniform(*d_range))
    L, R = _render(rng, W, H, boxes, d, 1.0, 10.0, 2.0)
    bx = np.array([b + [0] for b in boxes], dtype=np.int32).reshape(-1, 5)
    return Workload("pair640", [Frame(L, R)], bx, np.array(d, np.float32), dict(PARAMS["pair640"]))


def _random_frame(rng, W, H, n_obj, side_range, far_side, d_far, d_close, strip_frac):
    boxes, d = [], []
    for _ in range(n_obj):
        side = _loguniform(rng, *side_range)
        b = _box_of_side(rng, side, W, H)
        far = max(b[2] - b[0], b[3] - b[1]) < far_side
        boxes.append(b)
        d.append(rng.uniform(*(d_far if far else d_close)))
    n_base = len(boxes)
    for i in range(n_base):
        if strip_frac > 0 and rng.uniform() < strip_frac:
            x0, y0, x1, y1 = boxes[i]
            w = x1 - x0
            sw = max(2, int(round(rng.uniform(0.1, 0.3) * w)))
            sw = min(sw, w)
            sx0 = int(rng.integers(x0, x1 - sw + 1))
            dy = int(rng.integers(1, 11))
            boxes.append([sx0, y0, sx0 + sw, min(y1 + dy, H)])
            d.append(d[i] + rng.uniform(5.0, 20.0))
    return boxes, d


def multi_frame(name: str, seed: int, n_frames: int, W: int, H: int, boxes_per_frame,
                side_range, d_far, d_close, strip_frac: float = 0.0,
                gain_range=(0.8, 1.2), offset_range=(-20.0, 20.0), sigma: float = 2.0,
                poisson: bool = False, max_boxes: int | None = None) -> Workload:
    params = dict(PARAMS[name])

    def one(fi):
        rng = _frame_rng(seed, fi)
        n_obj = int(rng.poisson(boxes_per_frame)) if poisson else int(boxes_per_frame)
        if max_boxes is not None:
            n_obj = min(n_obj, max_boxes)
        boxes, d = _random_frame(rng, W, H, n_obj, side_range, params["far_side_px"],
                                 d_far, d_close, strip_frac)
        gain = rng.uniform(*gain_range)
        offset = rng.uniform(*offset_range)
        L, R = _render(rng, W, H, boxes, d, gain, offset, sigma)
        return Frame(L, R), boxes, d

    # every frame draws from its own generator, so frames can be made side by side
    # (numpy releases the interpreter lock) with the same result as in order
    workers = min(n_frames, os.cpu_count() or 1, 16)
    if workers > 1 and W * H >= 1 << 20:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            made = list(ex.map(one, range(n_frames)))
    else:
        made = [one(fi) for fi in range(n_frames)]
    frames, all_boxes, all_d = [], [], []
    for fi, (fr, boxes, d) in enumerate(made):
        frames.append(fr)
        all_boxes += [b + [fi] for b in boxes]
        all_d += d
    bx = np.array(all_boxes, dtype=np.int32).reshape(-1, 5)
    return Workload(name, frames, bx, np.array(all_d, np.float32), params)


def frame1080(seed: int = 1001, W: int = 1920, H: int = 1080, n_boxes: int = 64,
              side_range=(12.0, 400.0)) -> Workload:
    """One 1920x1080 frame, 64 boxes, far/close split (far d U[0.5,30], close U[2,250])."""
    return multi_frame("frame1080", seed, 1, W, H, n_boxes, side_range, (0.5, 30.0), (2.0, 250.0))


def batch32x1200(seed: int = 1002, n_frames: int = 32, W: int = 1920, H: int = 1200,
                 mean_boxes: float = 40.0, side_range=(12.0, 600.0)) -> Workload:
    """32 frames 1920x1200, Poisson(40) boxes, d_true U[0.5,120], 20% occluding strips."""
    return multi_frame("batch32x1200", seed, n_frames, W, H, mean_boxes, side_range,
                       (0.5, 120.0), (0.5, 120.0), strip_frac=0.2, poisson=True)


def batch8x2160(seed: int = 1003, n_frames: int = 8, W: int = 3840, H: int = 2160,
                n_boxes: int = 256, side_range=(12.0, 800.0)) -> Workload:
    """8 frames 3840x2160, 256 boxes each (far d U[0.5,60], close U[2,250])."""
    return multi_frame("batch8x2160", seed, n_frames, W, H, n_boxes, side_range,
                       (0.5, 60.0), (2.0, 250.0))


def by_name(name: str, **kw) -> Workload:
    return {"pair640": pair640, "frame1080": frame1080, "batch32x1200": batch32x1200,
            "batch8x2160": batch8x2160}[name](**kw)


# --------------------------------------------------------------------------- serving

SERVING_SIZES = ((1280, 720), (1920, 1080), (3840, 2160))


@dataclass
class ServingStream:
    width: int
    height: int
    frames: list     # Frame objects cycled through by the stream
    boxes: list      # int32 [n_i, 5] per frame (column 4 = 0)
    d_true: list


@dataclass
class ServingTrace:
    streams: list    # ServingStream per camera stream
    arrivals: list   # (t_s, stream, frame index within the stream's list), sorted by time
    params: dict


def serving(seed: int = 1004, n_streams: int = 4, rate_hz: float = 30.0, duration_s: float = 10.0,
            unique_frames: int = 3, jitter_ms: float = 5.0, mean_boxes: float = 60.0,
            max_boxes: int = 200, side_range=(12.0, 400.0), sizes=SERVING_SIZES,
            stream_sizes=None) -> ServingTrace:
    """Several stereo streams at a fixed rate: each stream's frame size is drawn
    once from `sizes`; each frame has min(max_boxes, Poisson(mean_boxes)) boxes
    (far d U[0.5,30], close U[2,250], gain/offset/noise as the 1080p frame);
    frame k of a stream arrives at k / rate + U[-jitter, +jitter] ms.  A stream
    cycles through `unique_frames` rendered frames.  `stream_sizes` fixes each
    stream's (width, height) instead of drawing it."""
    params = dict(PARAMS["serving"])
    top = np.random.Generator(np.random.PCG64([seed, 0xFFFF]))
    streams = []
    for s in range(n_streams):
        W, H = sizes[int(top.integers(0, len(sizes)))]
        if stream_sizes is not None:
            W, H = stream_sizes[s]
        frames, boxes, dts = [], [], []
        for k in range(unique_frames):
            rng = np.random.Generator(np.random.PCG64([seed, s, k]))
            n_obj = min(int(rng.poisson(mean_boxes)), max_boxes)
            bx, d = _random_frame(rng, W, H, n_obj, side_range, params["far_side_px"],
                                  (0.5, 30.0), (2.0, 250.0), 0.0)
            gain = rng.uniform(0.8, 1.2)
            offset = rng.uniform(-20.0, 20.0)
            L, R = _render(rng, W, H, bx, d, gain, offset, 2.0)
            frames.append(Frame(L, R))
            boxes.append(np.array([b + [0] for b in bx], dtype=np.int32).reshape(-1, 5))
            dts.append(np.array(d, np.float32))
        streams.append(ServingStream(W, H, frames, boxes, dts))
    arrivals = []
    n_per = int(round(rate_hz * duration_s))
    for s in range(n_streams):
        for k in range(n_per):
            t = k / rate_hz + top.uniform(-jitter_ms, jitter_ms) * 1e-3
            arrivals.append((max(t, 0.0), s, k % unique_frames))
    arrivals.sort()
    return ServingTrace(streams, arrivals, params)
