"""Mask post-pass: the 3 x 3 median filter kernel against the oracle's median
(Section 4: the BMC figure's median-filtered masks), bit for bit.

Sizes cover one-pixel-wide and one-pixel-high frames, widths below, at and
above one 32-bit word (rows that start mid-word and words that span several
rows), a ragged last word whose spare bits the input sets (they must be
ignored and come out clear), and the 1920 x 1080 x 200 mask the benchmark
filters, checked on sampled frames."""
import numpy as np
import pytest

from oracle import cdmd as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


@pytest.fixture(scope="module")
def ctx(C):
    return C.Context(0)


def _packed(mask, dirty_tail=True):
    words = O.pack_mask(mask)
    m = mask.shape[0]
    if dirty_tail and m % 32:
        words[:, -1] |= np.uint32(0xFFFFFFFF ^ ((1 << (m % 32)) - 1))
    return torch.from_numpy(words.view(np.int32)).cuda()


@pytest.mark.parametrize("W,H,n", [(1, 1, 3), (1, 45, 2), (45, 1, 2), (31, 9, 5), (32, 8, 4), (33, 7, 6),
                                   (61, 37, 9), (7, 200, 3), (320, 240, 5)])
@pytest.mark.parametrize("p", [0.3, 0.55])
def test_median_matches_oracle(C, ctx, W, H, n, p):
    m = W * H
    rng = np.random.default_rng(W * 1000 + H + int(p * 10))
    mask = rng.random((m, n)) < p
    out = C.cdmd_median3x3(ctx, _packed(mask), W, H)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    want = O.pack_mask(O.median3x3_mask(mask, W, H))
    assert np.array_equal(got, want)


def test_median_structured_mask(C, ctx):
    # blobs and speckle, as a thresholded frame has them: speckle goes, blobs stay
    W, H, n = 97, 53, 4
    m = W * H
    yy, xx = np.mgrid[0:H, 0:W]
    rng = np.random.default_rng(3)
    frames = []
    for t in range(n):
        f = ((xx - 20 - 5 * t) ** 2 + (yy - 25) ** 2 < 100) | (rng.random((H, W)) < 0.05)
        frames.append(f)
    mask = np.stack(frames).reshape(n, m).T
    got = C.unpack_mask(C.cdmd_median3x3(ctx, _packed(mask, dirty_tail=False), W, H), m)
    want = O.median3x3_mask(mask, W, H)
    assert np.array_equal(got, want)
    assert want.sum() < mask.sum()


def test_median_full_hd_sampled_frames(C, ctx):
    # the benchmark's launch: 1920 x 1080 x 200, one call; frames checked
    # against the oracle one by one (first, last and one in the middle)
    W, H, n = 1920, 1080, 200
    m = W * H
    g = torch.Generator(device="cuda").manual_seed(11)
    words = torch.randint(-2 ** 31, 2 ** 31 - 1, (n, (m + 31) // 32), dtype=torch.int32, device="cuda", generator=g)
    words &= torch.randint(-2 ** 31, 2 ** 31 - 1, words.shape, dtype=torch.int32, device="cuda", generator=g)
    out = C.cdmd_median3x3(ctx, words, W, H)
    torch.cuda.synchronize()
    for t in (0, 117, n - 1):
        frame = C.unpack_mask(words[t:t + 1].contiguous(), m)
        assert np.array_equal(C.unpack_mask(out[t:t + 1].contiguous(), m), O.median3x3_mask(frame, W, H))


def test_median_rejects_bad_arguments(C, ctx):
    mask = torch.zeros((2, 4), dtype=torch.int32, device="cuda")
    other = torch.zeros((2, 4), dtype=torch.int32, device="cuda")
    lib, h = ctx.lib, ctx.handle
    INVALID_ARG = next(k for k, v in C.STATUS_NAMES.items() if v == "CDMD_ERR_INVALID_ARG")
    ok = lib.cdmd_median3x3(h, mask.data_ptr(), 8, 16, 2, other.data_ptr(), None)
    assert ok == C.CDMD_OK
    bad = [(mask.data_ptr(), 8, 16, 2, mask.data_ptr()),            # in place
           (mask.data_ptr(), 8, 16, 2, mask.data_ptr() + 4),        # overlapping
           (mask.data_ptr(), 0, 16, 2, other.data_ptr()),           # W < 1
           (mask.data_ptr(), 8, 0, 2, other.data_ptr()),            # H < 1
           (mask.data_ptr(), 1 << 16, 1 << 16, 2, other.data_ptr()),  # W*H > 2^31 - 1
           (mask.data_ptr(), 8, 16, 0, other.data_ptr()),           # n < 1
           (mask.data_ptr() + 2, 8, 16, 2, other.data_ptr()),       # misaligned
           (None, 8, 16, 2, other.data_ptr())]
    for args in bad:
        assert lib.cdmd_median3x3(h, *args, None) == INVALID_ARG, args
    torch.cuda.synchronize()
    with pytest.raises(C.CdmdError):
        C.cdmd_median3x3(ctx, mask, 8, 16, out=mask)
    with pytest.raises(ValueError):
        C.cdmd_median3x3(ctx, mask, 9, 16)                        # words do not fit W*H
    with pytest.raises(ValueError):
        C.cdmd_median3x3(ctx, mask.float(), 8, 16)
