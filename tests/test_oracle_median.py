"""Pins for the oracle's 3 x 3 median filter of the mask (Section 4, the BMC
figure's median-filtered masks).

* scipy.ndimage.median_filter with a 3 x 3 window and constant zero padding
  computes the same filter by its own route (sorting the window).
* Brute force: pure-Python loops over each pixel's neighbours, on tiny frames.
* Closed forms: an all-ones frame keeps every pixel except its four corners
  (a corner sees 4 ones out of 9, an edge pixel 6); a single foreground pixel
  vanishes; a 3 x 3 block keeps its centre (9 ones) and edge midpoints
  (6 ones) and loses its corners (4 ones).
* Frames are filtered independently and pixel j sits at (j // W, j % W): a
  transposed layout or a row wrap (left neighbour taken from the previous
  row's end) fails the 1-pixel-wide and 1-pixel-high cases.
"""
import numpy as np
import pytest

from oracle import cdmd as O


def _brute(frame):
    H, W = frame.shape
    out = np.zeros_like(frame, dtype=bool)
    for y in range(H):
        for x in range(W):
            ones = 0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W and frame[yy, xx]:
                        ones += 1
            out[y, x] = ones >= 5
    return out


def _to_mask(frames):
    n, H, W = frames.shape
    return frames.reshape(n, H * W).T


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (2, 2), (5, 4), (9, 6)])
def test_median_matches_brute_force(W, H):
    rng = np.random.default_rng(W * 31 + H)
    frames = rng.random((3, H, W)) < 0.5
    got = O.median3x3_mask(_to_mask(frames), W, H)
    want = np.stack([_brute(f) for f in frames]).reshape(3, W * H).T
    assert np.array_equal(got, want)


@pytest.mark.parametrize("W,H,p", [(64, 48, 0.5), (33, 17, 0.3), (120, 5, 0.7)])
def test_median_matches_scipy(W, H, p):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(H)
    frames = rng.random((4, H, W)) < p
    got = O.median3x3_mask(_to_mask(frames), W, H)
    want = np.stack([ndimage.median_filter(f.astype(np.uint8), size=3, mode="constant", cval=0) for f in frames])
    assert np.array_equal(got, _to_mask(want.astype(bool)))


def test_median_all_ones_loses_only_corners():
    W, H = 11, 7
    got = O.median3x3_mask(np.ones((W * H, 2), dtype=bool), W, H).T.reshape(2, H, W)
    want = np.ones((H, W), dtype=bool)
    want[0, 0] = want[0, -1] = want[-1, 0] = want[-1, -1] = False
    assert np.array_equal(got[0], want) and np.array_equal(got[1], want)


def test_median_isolated_pixel_and_block():
    W, H = 9, 8
    f = np.zeros((H, W), dtype=bool)
    f[1, 1] = True                 # isolated: removed
    f[4:7, 4:7] = True             # 3 x 3 block: corners removed
    got = O.median3x3_mask(_to_mask(f[None]), W, H)[:, 0].reshape(H, W)
    want = np.zeros((H, W), dtype=bool)
    want[5, 4:7] = True
    want[4:7, 5] = True
    assert np.array_equal(got, want)


def test_median_thin_frames_do_not_wrap():
    # W = 1: every pixel's only neighbours are above and below
    col = np.array([1, 1, 0, 1, 1, 1, 0], dtype=bool)
    got = O.median3x3_mask(col[:, None], 1, 7)[:, 0]
    assert not got.any()           # at most 3 ones in any window
    # H = 2, W = 4, all ones: each pixel sees 4 (corner) or 6 (edge) ones
    got = O.median3x3_mask(np.ones((8, 1), dtype=bool), 4, 2)[:, 0].reshape(2, 4)
    assert np.array_equal(got, np.array([[0, 1, 1, 0], [0, 1, 1, 0]], dtype=bool))
