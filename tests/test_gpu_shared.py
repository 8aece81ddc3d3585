"""Clips that share one measurement matrix (same pixel count, k and seed):
cdmd_sketch_shared, cdmd_run_shared, cdmd_run_host_shared and the batch
plan's paired sketch items, against the FP64 oracle and against the per-clip
calls.

The mixed-precision sketch of a pair draws each entry of C once and applies
it to both clips' frames, so each clip's DY must be the oracle's C D_i to the
same tolerance as the per-clip mixed sketch, and agree with the per-clip
sketch up to the rounding order of the split sums."""
import numpy as np
import pytest

import videogen
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


def _padded(clip):
    """Device view (n, m) with row stride rounded up to 16 bytes and 255 in
    the bytes past m (which the kernels must not read)."""
    m, n = clip.m, clip.n
    ldd = (m + 15) // 16 * 16
    buf = np.full((n, ldd), 255, dtype=np.uint8)
    buf[:, :m] = clip.frames
    return torch.from_numpy(buf).cuda()[:, :m]


def _clips(w, h, ns, seed0):
    return [videogen.make_clip(w, h, n, seed=seed0 + i, drift=0.05) for i, n in enumerate(ns)]


# (w, h, frames of each clip, k): several row blocks and K steps, a ragged
# pixel count, rows not a multiple of 128, clips longer than 256 frames (cut
# into segments), five 200-frame clips (two packed launches, clips split
# across slots and launches), nine 16-frame clips (more segments than one
# launch takes), frame counts that are not multiples of 8 or 16
CASES = [(160, 120, (100, 120), 200), (97, 61, (37, 200), 203), (64, 33, (256, 128), 300),
         (384, 160, (200, 200), 1000), (300, 40, (16, 16), 513), (48, 32, (300, 40), 120),
         (80, 48, (240, 240), 96), (112, 80, (150, 61, 77), 260), (96, 64, (200,) * 5, 400),
         (64, 48, (16,) * 9, 64), (72, 40, (511, 3, 90), 130)]


@pytest.mark.parametrize("w,h,ns,k", CASES)
def test_sketch_shared_matches_oracle_and_solo(C, ctx, w, h, ns, k):
    clips = _clips(w, h, ns, seed0=31 * w + k)
    Ds = [_padded(c) for c in clips]
    m = clips[0].m
    seed = 777 + k
    DYs = C.cdmd_sketch_shared(ctx, Ds, k, seed, prec="bf16x2")
    C.cdmd_status_sync(ctx)
    Cm = M.measurement_matrix("gaussian", seed, k, m)
    for i, (clip, D, DY) in enumerate(zip(clips, Ds, DYs)):
        got = DY.cpu().numpy().T
        ref = O.sketch(Cm, clip.video_matrix())
        # BF16 hi + lo C and FP32 accumulation: the per-clip mixed bound
        err = np.abs(got - ref).max()
        assert err <= 1e-4 * np.sqrt(m) * 255.0, (i, err)
        solo = C.cdmd_sketch(ctx, D, k, seed, prec="bf16x2").cpu().numpy().T
        rel = np.linalg.norm(got - solo) / np.linalg.norm(solo)
        assert rel < 2e-5, (i, rel)


def test_sketch_shared_fp32_is_the_per_clip_sketch(C, ctx):
    clips = _clips(96, 64, (50, 70), seed0=5)
    Ds = [_padded(c) for c in clips]
    DYs = C.cdmd_sketch_shared(ctx, Ds, 150, 99, prec="fp32")
    for D, DY in zip(Ds, DYs):
        solo = C.cdmd_sketch(ctx, D, 150, 99, prec="fp32")
        assert torch.equal(DY, solo)


def test_sketch_shared_rejects_bad_arguments(C, ctx):
    clips = _clips(64, 48, (20, 20), seed0=1)
    Ds = [_padded(c) for c in clips]
    import ctypes
    arr = (ctypes.c_void_p * 1)()
    ns = (ctypes.c_int * 1)()
    ld = (ctypes.c_int64 * 1)()
    with pytest.raises(C.CdmdError, match="nclips"):
        C._check(ctx.lib.cdmd_sketch_shared(ctx.handle, 0, arr, 64 * 48, ns, ld, C.CTYPES["gaussian"], 10, 1,
                                            C.PRECS["bf16x2"], arr, None))
    with pytest.raises(ValueError, match="pixel count"):
        C.cdmd_sketch_shared(ctx, [Ds[0], _padded(videogen.make_clip(32, 48, 20, seed=2))], 10, 1, prec="bf16x2")
    odd = torch.from_numpy(np.zeros((20, 1001), dtype=np.uint8)).cuda()
    odd2 = torch.from_numpy(np.zeros((20, 1001), dtype=np.uint8)).cuda()
    with pytest.raises(C.CdmdError, match="16-byte"):
        C.cdmd_sketch_shared(ctx, [odd, odd2], 10, 1, prec="bf16x2")


def test_run_shared_matches_per_clip_runs(C, ctx):
    w, h, k, r, K = 240, 160, 400, 14, 8
    clips = _clips(w, h, (120, 150), seed0=71)
    Ds = [_padded(c) for c in clips]
    p = C.make_params(k, r, K, 25.0, seed=4711, prec="bf16x2", selector="omp")
    masks = C.cdmd_run_shared(ctx, Ds, p)
    C.cdmd_status_sync(ctx)
    m = clips[0].m
    for D, mk in zip(Ds, masks):
        solo = C.cdmd_run(ctx, D, p)
        C.cdmd_status_sync(ctx)
        a, b = C.unpack_mask(mk, m), C.unpack_mask(solo, m)
        # the shared sketch sums its splits in another order: decisions may
        # move only at pixels sitting on the threshold
        assert np.mean(a != b) <= 2e-4
    # the host-buffer form runs the same kernels on the same inputs
    hosts = [torch.from_numpy(c.frames).pin_memory() for c in clips]
    hm = C.cdmd_run_host_shared(ctx, hosts, p)
    dense = [torch.from_numpy(c.frames).cuda() for c in clips]
    dm = C.cdmd_run_shared(ctx, dense, p)
    C.cdmd_status_sync(ctx)
    for a, b in zip(hm, dm):
        assert torch.equal(a, b.cpu())


def test_run_shared_names_the_bad_clip(C, ctx):
    clips = _clips(64, 48, (40, 8), seed0=3)
    Ds = [_padded(c) for c in clips]
    p = C.make_params(100, 10, 5, 25.0, seed=1, prec="bf16x2", selector="omp")    # r = 10 > n - 1 = 7 for clip 1
    with pytest.raises(C.CdmdError, match="clip 1"):
        C.cdmd_run_shared(ctx, Ds, p)


def test_batch_pairs_clips_that_share_c(C):
    # one camera: every clip has the same pixel count, k and seed, so the
    # batch plan sketches them two at a time
    w, h, k, seed = 320, 192, 600, 1234
    clips = _clips(w, h, (100, 160, 90, 200, 61), seed0=900)
    cl = [dict(D=torch.from_numpy(c.frames).cuda(), k=k, r=16, K=10, seed=seed) for c in clips]
    ctx = C.Context(0)
    batch = C.Batch(cl, 25.0, prec="bf16x2", selector="omp", lanes=3)
    batch.run()
    batch.status_sync()
    Cm = M.measurement_matrix("gaussian", seed, k, clips[0].m)
    for i, (clip, c) in enumerate(zip(clips, cl)):
        v = batch.views(i)
        ref = O.sketch(Cm, clip.video_matrix())
        assert np.abs(v["DY"].T - ref).max() <= 1e-4 * np.sqrt(clip.m) * 255.0
        solo = C.cdmd_sketch(ctx, c["D"], k, seed, prec="bf16x2").cpu().numpy()
        assert np.linalg.norm(v["DY"] - solo) <= 2e-5 * np.linalg.norm(solo)
        mk = C.cdmd_run(ctx, c["D"], C.make_params(k, 16, 10, 25.0, seed=seed, prec="bf16x2", selector="omp"))
        C.cdmd_status_sync(ctx)
        a, b = C.unpack_mask(batch.masks[i], clip.m), C.unpack_mask(mk, clip.m)
        assert np.mean(a != b) <= 2e-4
    batch.close()
