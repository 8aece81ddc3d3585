"""Pass (a) with Rademacher C on the tensor cores (BF16X2 precision): the
per-clip launch (`cdmd_sketch`) and the packed launch of several clips under
one C (`cdmd_sketch_shared`) against the oracle's FP64 sketch with the same C.

+1 and -1 are exact in BF16, the pixels too, so every product is exact and
only the FP32 accumulation in tensor memory can round.  All partial sums are
integers bounded by 255 times the pixels summed; below 2^24 they are exact.
So for m < 65,793 pixels the sketch must equal the oracle's bit for bit,
whatever the split of the pixels over CTAs.  Above that the error of an
entry is bounded by (16-pixel additions + 1) 2^-23 times the sum of the
frame's pixels (the accumulation truncates; the running sum never exceeds
that sum in magnitude)."""
import numpy as np
import pytest

from oracle import cdmd as O
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


def _frames(n, m, seed):
    return np.random.default_rng(seed).integers(0, 256, size=(n, m), dtype=np.uint8)


def _oracle_dy(frames, k, seed):
    Cm = M.measurement_matrix("rademacher", seed, k, frames.shape[1])
    return O.sketch(Cm, frames.T.astype(np.float64)).T      # (n, k)


# (m, n, k): ragged pixel counts (not multiples of 64), k below, at and above
# one and two 128-row tiles, n odd, n = 256, and n > 256 (two launches)
CASES = [(2257, 30, 150), (5917, 200, 128), (4096, 256, 300), (1320, 77, 1000), (3001, 300, 64)]


@pytest.mark.parametrize("m,n,k", CASES)
def test_rademacher_tc_per_clip_is_exact(C, ctx, m, n, k):
    frames = _frames(n, m, m + n)
    ldd = (m + 15) // 16 * 16
    padded = np.full((n, ldd), 255, dtype=np.uint8)          # bytes past m must be ignored
    padded[:, :m] = frames
    D = torch.from_numpy(padded).cuda()[:, :m]
    DY = C.cdmd_sketch(ctx, D, k, 21 + k, ctype="rademacher", prec="bf16x2")
    C.cdmd_status_sync(ctx)
    assert np.array_equal(DY.cpu().numpy(), _oracle_dy(frames, k, 21 + k))


@pytest.mark.parametrize("ns", [[200, 200], [200, 200, 200, 200, 200], [31, 257, 90], [512, 3]])
def test_rademacher_tc_packed_is_exact(C, ctx, ns):
    m, k = 2992, 200            # a multiple of 16 (the BF16X2 path's row-stride rule), not of 64
    clips = [_frames(n, m, 100 + i) for i, n in enumerate(ns)]
    Ds = [torch.from_numpy(f).cuda() for f in clips]
    DYs = C.cdmd_sketch_shared(ctx, Ds, k, 99, ctype="rademacher", prec="bf16x2")
    C.cdmd_status_sync(ctx)
    Cm = M.measurement_matrix("rademacher", 99, k, m)
    for f, DY in zip(clips, DYs):
        assert np.array_equal(DY.cpu().numpy(), O.sketch(Cm, f.T.astype(np.float64)).T)


def test_rademacher_tc_matches_fp32_path(C, ctx):
    # the FP32 FMA path draws the same C (same counters): both are exact here
    m, n, k = 4976, 120, 260
    D = torch.from_numpy(_frames(n, m, 5)).cuda()
    a = C.cdmd_sketch(ctx, D, k, 8, ctype="rademacher", prec="bf16x2")
    b = C.cdmd_sketch(ctx, D, k, 8, ctype="rademacher", prec="fp32")
    C.cdmd_status_sync(ctx)
    assert torch.equal(a, b)


def test_rademacher_tc_full_hd_sampled_rows(C, ctx):
    # 1920 x 1080 x 200, k = 1000, packed with a second clip: sampled rows of
    # C against the oracle, within the truncation bound
    W, H, n, k = 1920, 1080, 200, 1000
    m = W * H
    g = torch.Generator(device="cuda").manual_seed(3)
    Ds = [torch.randint(0, 256, (n, m), dtype=torch.uint8, device="cuda", generator=g) for _ in range(2)]
    DYs = C.cdmd_sketch_shared(ctx, Ds, k, 12345, ctype="rademacher", prec="bf16x2")
    C.cdmd_status_sync(ctx)
    rows = np.array([0, 1, 127, 128, 500, 999])
    Cr = M.rademacher_block(12345, rows, np.arange(m))
    bound_steps = (m + 15) // 16 + 1
    for D, DY in zip(Ds, DYs):
        for t in (0, 77, n - 1):
            x = D[t].cpu().numpy().astype(np.float64)
            want = Cr @ x
            got = DY[t].cpu().numpy()[rows]
            assert np.all(np.abs(got - want) <= bound_steps * 2.0 ** -23 * x.sum()), (t, got - want)
            # far tighter in practice: the errors are a few ulps of the partial sums
            assert np.all(np.abs(got - want) <= 1e-6 * x.sum())


def test_run_with_rademacher_tc(C, ctx):
    # the whole pipeline takes the tensor-core Rademacher sketch
    import videogen
    clip = videogen.make_clip(96, 64, 80, seed=4)
    D = torch.from_numpy(clip.frames).cuda()
    k, r, K, tau, seed = 200, 10, 6, 25.0, 17
    mask = C.cdmd_run(ctx, D, C.make_params(k, r, K, tau, seed=seed, ctype="rademacher", prec="bf16x2"))
    DY = C.cdmd_sketch(ctx, D, k, seed, ctype="rademacher", prec="bf16x2")
    dec = C.cdmd_decompose(ctx, DY, r, K)
    Phi = C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K, prec="bf16x2")
    mask2 = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], tau, cols=dec["sel"])
    C.cdmd_status_sync(ctx)
    assert torch.equal(mask, mask2)
