"""GPU parity of the census kernel (Sec. 4.3.1) against the oracle: bit-exact."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.mark.parametrize("shape", [(5, 5), (37, 53), (480, 640), (121, 1923)])
@pytest.mark.parametrize("win", [(5, 5), (7, 7), (9, 7), (3, 5), (11, 3)])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_census_bit_exact(torch_cuda, shape, win, k):
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(hash((shape, win, k)) & 0xffff)
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    img[: shape[0] // 3, : shape[1] // 4] = 77  # flat region with ties
    for s in (0, 1):
        got = B.census_build(torch_cuda.from_numpy(img).cuda(), k, *win, s).cpu().numpy().view(np.uint64)
        ref = orc.census(img, k, *win, s)
        assert got.shape == ref.shape
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"mismatch at {bad[:5].tolist()}"


def test_census_fig2_patch(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    patch = np.array([[48, 72, 35, 91, 63], [85, 57, 44, 68, 29], [61, 93, 55, 37, 76],
                      [42, 66, 81, 50, 88], [73, 38, 59, 94, 46]], np.uint8)
    got = B.census_build(torch_cuda.from_numpy(patch).cuda(), 1, 5, 5, 1).cpu().numpy().view(np.uint64)
    assert int(got[2, 2]) == 0x2BD65B6
    assert int(got.sum() - got[2, 2]) == 0


def test_census_pitched_input(torch_cuda):
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(5)
    big = rng.integers(0, 256, size=(64, 200), dtype=np.uint8)
    t = torch_cuda.from_numpy(big).cuda()[:, 10:150]  # row pitch 200, width 140
    got = B.census_build(t, 1, 9, 7, 1).cpu().numpy().view(np.uint64)
    ref = orc.census(np.ascontiguousarray(big[:, 10:150]), 1, 9, 7, 1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("width", [201, 203, 206])
def test_census_word_loads_straddling_the_row_end(torch_cuda, k, width):
    """Aligned rows (pitch 208) whose width is not a multiple of the load word: the
    words that straddle the row end are read byte by byte, codes stay bit-exact."""
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(width * 10 + k)
    big = rng.integers(0, 256, size=(67, 208), dtype=np.uint8)
    img = big[:, :width]
    t = torch_cuda.from_numpy(big).cuda()[:, :width]
    for win in ((9, 7), (5, 5)):
        got = B.census_build(t, k, *win, 1).cpu().numpy().view(np.uint64)
        ref = orc.census(np.ascontiguousarray(img), k, *win, 1)
        assert np.array_equal(got, ref), (win, np.argwhere(got != ref)[:5].tolist())


@pytest.mark.parametrize("shape", [(70, 300), (9, 4099)])
@pytest.mark.parametrize("win", [(15, 3), (3, 15), (13, 3), (7, 9), (1, 1)])
@pytest.mark.parametrize("k", [1, 4, 8, 64])
def test_census_window_and_factor_limits(torch_cuda, shape, win, k):
    """The widest and tallest windows (15 px), 64-bit codes (7x9 plus the sentinel),
    the 1x1 window (the sentinel alone), and decimation factors up to the largest
    accepted (64), on a tall-enough image and on a 9-row strip 4099 px wide."""
    from paper_2604_07980_gb300 import binding as B
    rng = np.random.default_rng(shape[1] * 1000 + win[0] * 100 + win[1] * 10 + k)
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    img[:, : shape[1] // 5] = 200  # flat region with ties
    for s in (0, 1):
        got = B.census_build(torch_cuda.from_numpy(img).cuda(), k, *win, s).cpu().numpy().view(np.uint64)
        ref = orc.census(img, k, *win, s)
        assert got.shape == ref.shape
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"{win} k {k} sentinel {s}: mismatch at {bad[:5].tolist()}"
