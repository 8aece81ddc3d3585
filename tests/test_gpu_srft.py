"""GPU SRFT sketch (Section 3.3, C = R F D applied by a fast transform)
against the FP64 oracle's explicit C (oracle.measurement.srft_block).

Cases span: m with a large {2,3,5}-smooth divisor (the FFT passes: radix 4,
2, 3 and 5), m with none (61 x 97: FFT length 1, the twiddled sums alone),
odd k (last frequency keeps its real row), n not a multiple of the frames a
CTA takes, a row stride ldd > m, and the 720x480 x 200 study size.  The
kept frequencies must equal the oracle's exactly; the sketch is FP32
arithmetic (FFT, hardware-accurate sine/cosine of exactly reduced phases)
with FP64 sums of the column-group partials, held to 2e-6 sqrt(m) 255
absolute (the FP32 sketch tests' scale) and the error is printed.
"""
import numpy as np
import pytest

import videogen
from oracle import measurement as M

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


@pytest.mark.parametrize("w,h,n,k,seed,pad", [(60, 48, 37, 7, 3, 0), (61, 97, 12, 40, 5, 0),
                                              (160, 120, 100, 200, 9, 16), (320, 240, 33, 1000, 1, 0),
                                              (99, 1, 5, 10, 2, 3)])
def test_srft_sketch_matches_oracle(C, ctx, w, h, n, k, seed, pad):
    clip = videogen.make_clip(w, h, n, seed=seed)
    m = clip.m
    frames = np.zeros((n, m + pad), dtype=np.uint8)
    frames[:, :m] = clip.frames
    Dfull = torch.from_numpy(frames).cuda()
    D = Dfull[:, :m]                                   # row stride m + pad
    meas = C.Measure(ctx, "srft", m, k, seed)
    np.testing.assert_array_equal(meas.rows.cpu().numpy(), M.srft_frequencies(seed, k, m))
    DY = C.cdmd_sketch_gather(ctx, D, meas)
    C.cdmd_status_sync(ctx)
    ref = M.srft_block(seed, np.arange(k), np.arange(m), m, k) @ clip.video_matrix()    # (k, n)
    err = np.abs(DY.cpu().numpy().T - ref)
    bound = 2e-6 * np.sqrt(m) * 255.0
    print(f"\nSRFT {w}x{h}x{n} k={k}: max abs err {err.max():.3e} (bound {bound:.3e}), "
          f"max |DY| {np.abs(ref).max():.3e}")
    assert err.max() <= bound


def test_srft_sketch_study_size_sampled_rows(C, ctx):
    w, h, n, k, seed = 720, 480, 200, 1000, 21
    clip = videogen.make_clip(w, h, n, seed=31)
    m = clip.m
    meas = C.Measure(ctx, "srft", m, k, seed)
    DY = C.cdmd_sketch_gather(ctx, torch.from_numpy(clip.frames).cuda(), meas)
    C.cdmd_status_sync(ctx)
    rows = np.array([0, 1, 2, 3, 500, 501, 998, 999])
    ref = M.srft_block(seed, rows, np.arange(m), m, k) @ clip.video_matrix()
    err = np.abs(DY.cpu().numpy().T[rows] - ref)
    bound = 2e-6 * np.sqrt(m) * 255.0
    print(f"\nSRFT 720x480x200 k=1000, sampled rows: max abs err {err.max():.3e} (bound {bound:.3e})")
    assert err.max() <= bound


def test_srft_build_rejects_bad_arguments(C, ctx):
    with pytest.raises(C.CdmdError):
        C.Measure(ctx, "srft", 10, 30, 1)           # ceil(k/2) = 15 > m
