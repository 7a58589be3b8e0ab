"""Independent brute-force restatements used to pin the oracle on tiny inputs.

These are deliberately different formulations from the oracle's loops: the
census is built from whole-array shifted comparisons weighted by powers of two,
the popcount goes through ``np.unpackbits`` and costs are gathered for every
candidate at once.  They are only fast enough for tiny images.
"""
from __future__ import annotations

import numpy as np


def census_np(img: np.ndarray, win_w: int, win_h: int, sentinel: int = 1) -> np.ndarray:
    """Census by array shifts: bit weight 2^(n-1-t) for the t-th window offset in
    raster order (Fig. 2's printed order), sentinel 2^n; undefined border -> 0."""
    img = img.astype(np.int64)
    H, W = img.shape
    sx, sy = win_w // 2, win_h // 2
    n = win_w * win_h
    code = np.zeros((H, W), dtype=object)
    code[:, :] = 0
    out = np.zeros((H, W), dtype=np.uint64)
    if H - 2 * sy <= 0 or W - 2 * sx <= 0:
        return out
    centre = img[sy:H - sy, sx:W - sx]
    acc = np.zeros(centre.shape, dtype=np.uint64)
    t = 0
    for j in range(-sy, sy + 1):
        for i in range(-sx, sx + 1):
            nb = img[sy + j:H - sy + j, sx + i:W - sx + i]
            acc |= (nb > centre).astype(np.uint64) << np.uint64(n - 1 - t)
            t += 1
    if sentinel:
        acc |= np.uint64(1) << np.uint64(n)
    out[sy:H - sy, sx:W - sx] = acc
    return out


def popcount_u64(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    bits = np.unpackbits(a.view(np.uint8).reshape(a.shape + (8,)), axis=-1)
    return bits.sum(axis=-1).astype(np.int64)


def shifted(c: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """out[y, x] = c[y + dy, x + dx] with zeros outside."""
    H, W = c.shape
    out = np.zeros_like(c)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    if ys1 > ys0 and xs1 > xs0:
        out[ys0:ys1, xs0:xs1] = c[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return out


def cost_volume(CL, CR, mask, dmin, dmax, dy_min, dy_max) -> np.ndarray:
    """S[dy, d] = sum over mask of popcount(CL ^ CR shifted to (x - d, y + dy))."""
    out = np.zeros((dy_max - dy_min + 1, dmax - dmin + 1), dtype=np.int64)
    for a, dy in enumerate(range(dy_min, dy_max + 1)):
        for b, d in enumerate(range(dmin, dmax + 1)):
            out[a, b] = popcount_u64((CL ^ shifted(CR, -d, dy))[mask]).sum()
    return out


def longest_run_median(vals, tau, nmin, mode=0, trim=0.2):
    """Brute force over every contiguous window of the sorted list."""
    v = np.sort(np.asarray(vals, dtype=np.float32))
    n = len(v)
    best = None
    for s in range(n):
        for e in range(s + 1, n + 1):
            w = v[s:e]
            ok = all((w[i + 1] - w[i]) < np.float32(tau) for i in range(len(w) - 1))
            if ok and (best is None or len(w) > len(best)):
                best = w
    if best is None or len(best) < nmin:
        return None
    return best
