"""The allocation-free sketch agrees with the context-based sketch.

cdmd_sketch_noalloc is for callers that cannot allocate device memory once
running (fixed start-up memory budgets, real-time or certified pipelines,
hosts whose allocator belongs to another runtime): its partial sums live in a
fixed array inside the library.  Two calls in a row, the first larger than
the second, must each match cdmd_sketch within the tolerance of the FP32
sketch tests; the second call reuses the array the first one filled.  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import videogen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


def test_noalloc_sketch_matches_cdmd_sketch_on_two_calls(C):
    ctx = C.Context(0)
    torch.cuda.set_device(0)
    cases = [((160, 120, 100), 200, "gaussian", 17), ((97, 61, 37), 203, "gaussian", 5)]
    for (w, h, n), k, ctype, seed in cases:
        clip = videogen.make_clip(w, h, n, seed=seed)
        D = torch.from_numpy(clip.frames).cuda()
        ref = C.cdmd_sketch(ctx, D, k, seed, ctype=ctype)
        got = C.cdmd_sketch_noalloc(D, k, seed, ctype=ctype)
        torch.cuda.synchronize()
        tol = 2e-6 * np.sqrt(clip.m) * 255.0
        assert (got - ref).abs().max().item() <= tol


def test_noalloc_sketch_at_the_array_limit_and_past_256_frames(C):
    """k n close to the array's 4,194,304 partial sums, so the split count is
    capped to one or two pixel ranges, and clips longer than 256 frames, which
    are sketched in 256-frame slabs that share the array; each case twice."""
    ctx = C.Context(0)
    torch.cuda.set_device(0)
    cases = [((64, 48, 4000), 1024, 23),      # k n = 4,096,000: one split fits
             ((96, 40, 2000), 2000, 29),      # k n = 4,000,000 over 3,840 pixels
             ((80, 60, 600), 300, 31)]        # three slabs, several splits
    for (w, h, n), k, seed in cases:
        clip = videogen.make_clip(w, h, n, seed=seed, n_objects=2)
        D = torch.from_numpy(clip.frames).cuda()
        ref = C.cdmd_sketch(ctx, D, k, seed)
        # with one or two splits a partial sum adds up to m FP32 products in
        # one chain, whose rounding walks about sqrt(m) 2^-24 of the sum's
        # size; the context sketch splits the pixels finer
        tol = 2e-6 * np.sqrt(clip.m) * 255.0 + 3.0 * np.sqrt(clip.m) * 2.0 ** -24 * ref.abs().max().item()
        for _ in range(2):
            got = C.cdmd_sketch_noalloc(D, k, seed)
            torch.cuda.synchronize()
            assert (got - ref).abs().max().item() <= tol


def test_noalloc_sketch_rademacher_is_exact_twice(C):
    ctx = C.Context(0)
    clip = videogen.make_clip(97, 61, 37, seed=5)
    D = torch.from_numpy(clip.frames).cuda()
    ref = C.cdmd_sketch(ctx, D, 130, 99, ctype="rademacher")
    for _ in range(2):
        got = C.cdmd_sketch_noalloc(D, 130, 99, ctype="rademacher")
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_sketch_rejects_sizes_beyond_its_array(C):
    D = torch.zeros((3000, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(C.CdmdError) as e:
        C.cdmd_sketch_noalloc(D, 1500, 1)        # k * n = 4.5e6 > 4,194,304
    assert e.value.status == 1
