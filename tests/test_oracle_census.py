"""Pins for the oracle's census (Sec. 4.3.1, Algorithm 1, Fig. 2)."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from tests.brute import census_np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig2_census.txt")


def _read_fig2():
    patch, code, mode = [], [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("patch", "code"):
            mode = line
            continue
        (patch if mode == "patch" else code).append(line.split())
    return np.array(patch, dtype=np.uint8), code


def test_fig2_worked_example():
    """The oracle's code for Fig. 2's patch equals the bits the figure prints."""
    patch, rows = _read_fig2()
    bits = "".join("0" if b == "." else b for row in rows for b in row)
    assert len(bits) == 25
    expected = int("1" + bits, 2)  # Algorithm 1: sentinel first, then the 25 bits
    c = orc.census(patch, k=1, win_w=5, win_h=5, sentinel=1)
    assert int(c[2, 2]) == expected == 0x2BD65B6
    c0 = orc.census(patch, k=1, win_w=5, win_h=5, sentinel=0)
    assert int(c0[2, 2]) == int(bits, 2)
    # only the centre pixel has its whole window inside the 5x5 patch
    m = np.ones((5, 5), bool)
    m[2, 2] = False
    assert np.all(c[m] == 0)


def test_fig2_colour_rule_strict_greater():
    """Fig. 2's legend: > centre -> 1, <= centre -> 0 (a neighbour equal to 55 gives 0)."""
    patch, _ = _read_fig2()
    p = patch.copy()
    p[0, 0] = 55
    c = int(orc.census(p, 1, 5, 5, 1)[2, 2])
    assert (c >> 24) & 1 == 0
    p[0, 0] = 56
    c = int(orc.census(p, 1, 5, 5, 1)[2, 2])
    assert (c >> 24) & 1 == 1


@pytest.mark.parametrize("win", [(5, 5), (7, 7), (9, 7)])
@pytest.mark.parametrize("sentinel", [0, 1])
def test_constant_image_is_all_zero(win, sentinel):
    img = np.full((23, 31), 117, np.uint8)
    c = orc.census(img, 1, *win, sentinel)
    n = win[0] * win[1]
    cmp_mask = np.uint64((1 << n) - 1)
    assert np.all((c & cmp_mask) == 0)
    sx, sy = win[0] // 2, win[1] // 2
    inner = c[sy:23 - sy, sx:31 - sx]
    assert np.all(inner == (np.uint64(1 << n) if sentinel else 0))


@pytest.mark.parametrize("win", [(3, 3), (5, 5), (7, 7), (9, 7), (3, 5)])
def test_brute_force_tiny(win):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(19, 26), dtype=np.uint8)
    img[3:9, 4:10] = 80  # a flat patch with ties
    for s in (0, 1):
        assert np.array_equal(orc.census(img, 1, *win, s), census_np(img, *win, s))


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("shape", [(24, 30), (25, 31)])
def test_scaled_census_is_census_of_decimated_image(k, shape):
    """Multi-resolution census (Sec. 4.3.1): equals the census of I[::k, ::k]."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    got = orc.census(img, k, 7, 7, 1)
    ref = census_np(np.ascontiguousarray(img[::k, ::k]), 7, 7, 1)
    assert got.shape == ref.shape == (-(-shape[0] // k), -(-shape[1] // k))
    assert np.array_equal(got, ref)


def test_offset_and_monotonic_invariance():
    """Census depends only on the order of intensities (Sec. 1, Sec. 4.3.1)."""
    rng = np.random.default_rng(3)
    img = rng.integers(0, 200, size=(30, 40), dtype=np.uint8)
    base = orc.census(img, 1, 9, 7, 1)
    assert np.array_equal(base, orc.census((img + 55).astype(np.uint8), 1, 9, 7, 1))
    v = np.arange(256)
    lut = np.clip(v + v // 4, 0, 255).astype(np.uint8)  # strictly increasing on 0..199
    assert np.all(np.diff(lut[:200].astype(int)) > 0)
    assert np.array_equal(base, orc.census(lut[img], 1, 9, 7, 1))
