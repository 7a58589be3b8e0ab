"""Pins of the oracle's Sec. 4.3.6 step (Q reprojection, vehicle transform) and
of the depth-variance equation, against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import oracle as orc

F, B = 2000.0, 0.30
CX, CY = 960.0, 600.0


def _q(cx=CX, cy=CY, f=F, b=B, cx2=CX):
    # reprojection matrix of a rectified pair (principal points cx, cx2 of the two cameras)
    return np.array([[1, 0, 0, -cx], [0, 1, 0, -cy], [0, 0, 0, f], [0, 0, 1 / b, (cx - cx2) / b]], float)


def _geo(Q=None, T=None, var=0.25, w=1920, h=1200):
    return dict(Q=_q() if Q is None else Q, T=np.hstack([np.eye(3), np.zeros((3, 1))]) if T is None else T,
                disp_var=var, f_px=F, baseline_m=B, width=w, height=h)


def _random_boxes(rng, n, W=1920, H=1200):
    x0 = rng.integers(0, W - 50, n)
    y0 = rng.integers(0, H - 50, n)
    w = rng.integers(2, 50, n)
    h = rng.integers(2, 50, n)
    return np.stack([x0, y0, x0 + w, y0 + h, np.zeros(n, int)], 1).astype(np.int32)


def test_standard_q_closed_form_and_eq1():
    rng = np.random.default_rng(7)
    boxes = _random_boxes(rng, 200)
    disp = rng.uniform(0.5, 250.0, 200).astype(np.float32)
    out = orc.box_points(boxes, disp, np.ones(200, np.uint8), [_geo()])
    u = (boxes[:, 0] + boxes[:, 2] - 1) / 2.0
    v = (boxes[:, 1] + boxes[:, 3] - 1) / 2.0
    d = disp.astype(np.float64)
    np.testing.assert_allclose(out[:, 0], (u - CX) * B / d, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[:, 1], (v - CY) * B / d, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[:, 2], F * B / d, rtol=1e-12)
    # Z is Eq. 1's depth (the oracle's fp32 Eq. 1 within fp32 rounding)
    z1 = np.array([orc.depth(F, B, float(x)) for x in disp])
    np.testing.assert_allclose(out[:, 2], z1, rtol=2e-7)
    np.testing.assert_allclose(out[:, 7], d / B, rtol=1e-12)


def test_variance_is_squared_depth_derivative():
    """sigma_Z^2 = (dZ/dd)^2 sigma_d^2, the derivative taken by central differences."""
    rng = np.random.default_rng(8)
    boxes = _random_boxes(rng, 50)
    disp = rng.uniform(2.0, 200.0, 50)
    var = 0.37
    g = [_geo(var=var)]
    out = orc.box_points(boxes, disp.astype(np.float32), np.ones(50, np.uint8), g)
    d32 = disp.astype(np.float32).astype(np.float64)
    h = 1e-3 * d32
    zp = orc.box_points(boxes, (d32 + h).astype(np.float32), np.ones(50, np.uint8), g)[:, 2]
    zm = orc.box_points(boxes, (d32 - h).astype(np.float32), np.ones(50, np.uint8), g)[:, 2]
    dd = (d32 + h).astype(np.float32).astype(np.float64) - (d32 - h).astype(np.float32).astype(np.float64)
    deriv = (zp - zm) / dd
    np.testing.assert_allclose(out[:, 6], deriv ** 2 * var, rtol=1e-5)


def test_vehicle_transform():
    rng = np.random.default_rng(9)
    boxes = _random_boxes(rng, 40)
    disp = rng.uniform(1.0, 100.0, 40).astype(np.float32)
    ident = orc.box_points(boxes, disp, np.ones(40, np.uint8), [_geo()])
    np.testing.assert_array_equal(ident[:, 3:6], ident[:, 0:3])
    # rotation by 90 degrees about the optical axis, then a translation
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float)
    t = np.array([1.5, -2.0, 0.25])
    out = orc.box_points(boxes, disp, np.ones(40, np.uint8), [_geo(T=np.hstack([R, t[:, None]]))])
    p = out[:, 0:3]
    np.testing.assert_allclose(out[:, 3], -p[:, 1] + t[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 4], p[:, 0] + t[1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 5], p[:, 2] + t[2], rtol=0, atol=1e-12)
    # a rigid transform keeps distances between points
    dc = np.linalg.norm(p[1:] - p[:-1], axis=1)
    dv = np.linalg.norm(out[1:, 3:6] - out[:-1, 3:6], axis=1)
    np.testing.assert_allclose(dv, dc, rtol=1e-12)


def test_homogeneous_scale_invariance_and_principal_point_shift():
    rng = np.random.default_rng(10)
    boxes = _random_boxes(rng, 30)
    disp = rng.uniform(1.0, 100.0, 30).astype(np.float32)
    a = orc.box_points(boxes, disp, np.ones(30, np.uint8), [_geo()])
    b = orc.box_points(boxes, disp, np.ones(30, np.uint8), [_geo(Q=-3.5 * _q())])
    np.testing.assert_allclose(b[:, :7], a[:, :7], rtol=1e-12, atol=1e-12)
    # different principal points: Z = f b / (d - (cx - cx'))
    c = orc.box_points(boxes, disp, np.ones(30, np.uint8), [_geo(Q=_q(cx2=CX - 4.0))])
    np.testing.assert_allclose(c[:, 2], F * B / (disp.astype(np.float64) + 4.0), rtol=1e-12)


def test_invalid_cases_are_nan_and_boxes_are_clipped():
    boxes = np.array([[10, 10, 30, 30, 0], [10, 10, 30, 30, 1], [10, 10, 30, 30, -1],
                      [-20, -40, 21, 11, 0], [1900, 1190, 2000, 1300, 0]], np.int32)
    disp = np.array([5, 5, 5, 5, 5], np.float32)
    flags = np.array([0x80, 1, 1, 1, 1], np.uint8)  # box 0 not VALID
    out = orc.box_points(boxes, disp, flags, [_geo()])
    assert np.isnan(out[0]).all()        # not VALID
    assert np.isnan(out[1]).all()        # no geometry for frame 1
    assert np.isnan(out[2]).all()        # negative frame index
    # clipped to [0, 21) x [0, 11): centre (10, 5)
    assert out[3, 0] == pytest.approx((10 - CX) * B / 5) and out[3, 1] == pytest.approx((5 - CY) * B / 5)
    # clipped to [1900, 1920) x [1190, 1200): centre (1909.5, 1194.5)
    assert out[4, 0] == pytest.approx((1909.5 - CX) * B / 5)
    # W == 0 (disparity 0 with the standard Q)
    z = orc.box_points(boxes[:1], np.zeros(1, np.float32), np.ones(1, np.uint8), [_geo()])
    assert np.isnan(z).all()
    assert math.isnan(orc.box_points(boxes[:1], disp[:1], np.ones(1, np.uint8), [_geo(Q=np.zeros((4, 4)))])[0, 0])
