"""Sec. 5.1 auto-rectification: the library's host filter against the oracle's
(CPU), and the device offset search against the oracle (GPU): counts are
integers and must be equal."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_07980_gb300 import workloads as wl


def test_rect_filter_matches_oracle():
    from paper_2604_07980_gb300 import binding as B
    try:
        B.lib()
    except B.CtmError:
        pytest.skip("library not built")
    rng = np.random.default_rng(31)
    for _ in range(500):
        n = int(rng.integers(0, 9))
        est = rng.integers(-6, 7, n)
        prev = int(rng.integers(-4, 5))
        step = int(rng.integers(0, 4))
        assert B.rect_filter(est, prev, step) == orc.rect_filter(est, prev, step)


@pytest.mark.gpu
def test_auto_rect_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(32)
    H, W, d_true = 120, 400, 17
    cases = []
    for delta_true in (-2, 3):
        big = np.clip(np.rint(wl.texture(rng, H + 12, W + 30)), 0, 255).astype(np.uint8)
        L = big[6:6 + H, :W].copy()
        R = big[6 + delta_true:6 + delta_true + H, d_true:d_true + W].copy()
        cases.append((L, R, (20, 8, 380, 110), 0, 63, -4, 4, 4, delta_true))
    noise = rng.integers(0, 256, (H, W), dtype=np.uint8)
    cases.append((noise, np.roll(noise, 5, axis=1), (0, 0, W, H), -3, 20, -1, 1, 0, None))  # borders, negative d
    for L, R, roi, dmin, dmax, dlo, dhi, thr, delta_true in cases:
        ref_best, ref_counts = orc.auto_rect(L, R, roi, dmin, dmax, dlo, dhi, thr)
        delta, counts = B.auto_rect(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), roi, dmin, dmax,
                                    dlo, dhi, thr)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy(), ref_counts)
        assert int(delta.item()) == ref_best
        if delta_true is not None:
            assert ref_best == delta_true
