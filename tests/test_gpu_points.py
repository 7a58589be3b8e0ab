"""ctm_box_points (Sec. 4.3.6 reprojection, vehicle transform, depth variance)
against the oracle, on the outputs of a matched batch: fp32 on the device vs
float64 in the oracle, with tolerances from fp32 rounding (a few ulp per
operation, a dozen operations)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _geometries(rng, n, W, H, f, b):
    out = []
    for _ in range(n):
        cx, cy = W / 2 + rng.uniform(-20, 20), H / 2 + rng.uniform(-20, 20)
        cx2 = cx + rng.uniform(-3, 3)
        Q = np.array([[1, 0, 0, -cx], [0, 1, 0, -cy], [0, 0, 0, f], [0, 0, 1 / b, (cx - cx2) / b]])
        a, c = rng.uniform(-0.3, 0.3, 2)
        Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
        Rx = np.array([[1, 0, 0], [0, np.cos(c), -np.sin(c)], [0, np.sin(c), np.cos(c)]])
        T = np.hstack([Rz @ Rx, rng.uniform(-2, 2, (3, 1))])
        out.append(dict(Q=Q.astype(np.float32), T=T.astype(np.float32), disp_var=0.25, f_px=f,
                        baseline_m=b, width=W, height=H))
    return out


def test_box_points_match_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    w = wl.batch32x1200(n_frames=4)
    ctx = B.Context(w.params, len(w.frames), 1920, 1200, w.n_boxes)
    batch = B.DeviceBatch(B.frames_to_device(w.frames), w.boxes, [(f.f_px, f.baseline_m) for f in w.frames])
    res = ctx.match_batch(batch, use_graph=False)
    rng = np.random.default_rng(11)
    geos = _geometries(rng, len(w.frames), 1920, 1200, wl.F_PX, wl.BASELINE_M)
    geo_dev, n_geo = B.geometries_to_device(geos)
    got = B.box_points(batch.boxes, res["disp"], res["flags"], geo_dev, n_geo).cpu().numpy()
    disp = res["disp"].cpu().numpy()
    flags = res["flags"].cpu().numpy()
    ref = orc.box_points(w.boxes, disp, flags, [dict(g, Q=g["Q"].astype(np.float64),
                                                    T=g["T"].astype(np.float64)) for g in geos])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref[:, 0])
    assert ok.sum() > 100
    scale = np.linalg.norm(ref[ok, 0:3], axis=1)[:, None] + 1.0
    err = np.abs(got[ok, 0:6] - ref[ok, 0:6])
    np.testing.assert_array_less(err, np.broadcast_to(4e-6 * scale + 1e-12, err.shape))
    np.testing.assert_allclose(got[ok, 6], ref[ok, 6], rtol=2e-5)
    np.testing.assert_allclose(got[ok, 7], ref[ok, 7], rtol=2e-6)
    # boxes given a frame index without geometry get NaN
    bad = batch.boxes.clone()
    bad[:, 4] = n_geo
    assert torch.isnan(B.box_points(bad, res["disp"], res["flags"], geo_dev, n_geo)).all()
    ctx.close()
