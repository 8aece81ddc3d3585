"""Exact DMD on the GPU (Section 2.1, the comparator of Section 4's
Computational Performance): the snapshot Gram pass against exact integer
inner products, the decomposition from a Gram against the one from a sketch,
and the whole exact-DMD pipeline against the FP64 oracle's exact DMD.

The Gram's products are exact (uint8 in FP16) and its sums accumulate in
FP32 over each CTA's pixel range.  The tensor cores' accumulation is not
rounded to nearest: an addition may lose up to one unit in the last place,
2^-23 of the running sum, and the losses add up coherently.  Every partial
is a sum of non-negative terms, so the running sum never exceeds the final
entry and an entry's error is bounded by (additions per CTA + 1) 2^-23 R.  Downstream the
pipeline is held to the mixed-precision bar: background within 1e-3 relative
of the oracle, F-measure within 0.001."""
import numpy as np
import pytest

import videogen
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


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _gram_bound(m, sms):
    steps = (m + 63) // 64
    per_cta = -(-steps // min(sms, steps))
    return (4 * per_cta + 1) * 2.0 ** -23


# (W, H, n): a pixel count that is not a multiple of 64, the smallest n, one
# and two 128-frame tiles and the boundary between them, the largest n
CASES = [(61, 37, 2), (61, 37, 17), (64, 48, 128), (64, 48, 129), (97, 61, 200), (40, 33, 256), (300, 41, 64)]


@pytest.mark.parametrize("W,H,n", CASES)
def test_snapshot_gram_matches_exact_integers(C, ctx, W, H, n):
    m = W * H
    rng = np.random.default_rng(W + n)
    frames = rng.integers(0, 256, size=(n, m), dtype=np.uint8)
    ldd = (m + 15) // 16 * 16
    padded = np.full((n, ldd), 255, dtype=np.uint8)          # bytes past m must be ignored
    padded[:, :m] = frames
    D = torch.from_numpy(padded).cuda()[:, :m]
    R = C.cdmd_snapshot_gram(ctx, D)
    C.cdmd_status_sync(ctx)
    R = R.cpu().numpy()
    exact = O.snapshot_gram(frames.T)
    assert np.array_equal(R, R.T)
    err = np.abs(R - exact.astype(np.float64))
    assert np.all(err <= _gram_bound(m, _sms()) * exact + 0.5), err.max()


def test_snapshot_gram_long_chains(C):
    # 4 SMs: every CTA accumulates ~300 K steps of 64 pixels in FP32
    cx = C.Context(0)
    C.cdmd_set_sm_limit(cx, 4)
    W, H, n = 320, 240, 100
    m = W * H
    frames = np.random.default_rng(9).integers(0, 256, size=(n, m), dtype=np.uint8)
    R = C.cdmd_snapshot_gram(cx, torch.from_numpy(frames).cuda())
    C.cdmd_status_sync(cx)
    exact = O.snapshot_gram(frames.T)
    err = np.abs(R.cpu().numpy() - exact)
    assert np.all(err <= _gram_bound(m, 4) * exact), (err / exact).max()


def test_snapshot_gram_full_hd_sampled(C, ctx):
    # the full-size launch (1920 x 1080 x 200); sampled entries exactly
    W, H, n = 1920, 1080, 200
    m = W * H
    g = torch.Generator(device="cuda").manual_seed(5)
    D = torch.randint(0, 256, (n, m), dtype=torch.uint8, device="cuda", generator=g)
    R = C.cdmd_snapshot_gram(ctx, D)
    C.cdmd_status_sync(ctx)
    R = R.cpu().numpy()
    assert np.array_equal(R, R.T)
    pairs = [(0, 0), (0, 199), (17, 130), (127, 128), (128, 128), (199, 199), (64, 3), (150, 151)]
    bound = _gram_bound(m, _sms())
    for s, t in pairs:
        a = D[s].cpu().numpy().astype(np.int64)
        b = D[t].cpu().numpy().astype(np.int64)
        exact = float(a @ b)
        assert abs(R[s, t] - exact) <= bound * exact, (s, t, R[s, t], exact)


@pytest.mark.parametrize("selector", ["omp", "lstsq"])
def test_decompose_gram_equals_decompose_of_sketch(C, ctx, selector):
    # decompose_gram on R = DY^T DY repeats cdmd_decompose on DY
    clip = videogen.make_clip(96, 64, 80, seed=2)
    D = torch.from_numpy(clip.frames).cuda()
    r, K = 12, 5
    DY = C.cdmd_sketch(ctx, D, 150, 41)
    ref = C.cdmd_decompose(ctx, DY, r, K, selector=selector)
    R = (DY @ DY.T).contiguous()
    got = C.cdmd_decompose_gram(ctx, R, r, K, selector=selector)
    C.cdmd_status_sync(ctx)
    lam_ref = ref["lam"].cpu().numpy()
    lam = got["lam"].cpu().numpy()
    scale = np.abs(lam_ref[:, 0] + 1j * lam_ref[:, 1]).max()
    assert np.abs(lam - lam_ref).max() <= 1e-8 * scale
    assert torch.equal(got["sel"], ref["sel"]) and torch.equal(got["nsel"], ref["nsel"])
    b_ref = ref["beta"].cpu().numpy()
    assert np.abs(got["beta"].cpu().numpy() - b_ref).max() <= 1e-6 * np.abs(b_ref).max()


@pytest.mark.parametrize("seed,prec", [(3, "bf16x2"), (4, "fp32")])
def test_exact_dmd_pipeline_matches_oracle(C, ctx, seed, prec):
    clip = videogen.make_clip(160, 120, 100, seed=seed)
    r, K, tau = 10, 6, 25.0
    Dm = clip.video_matrix()
    ref = O.exact_dmd(Dm, r, K)
    ref_bg = O.background(ref["Phi"][:, ref["sel"]], ref["beta"], ref["lam"][ref["sel"]], clip.n)
    D = torch.from_numpy(clip.frames).cuda()
    R = C.cdmd_snapshot_gram(ctx, D)
    dec = C.cdmd_decompose_gram(ctx, R, r, K)
    Phi = C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K, prec=prec)
    mask, bg = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], tau, cols=dec["sel"], want_bg=True)
    C.cdmd_status_sync(ctx)
    # the selected modes and their eigenvalues
    sel = dec["sel"].cpu().numpy()
    assert set(sel.tolist()) == set(int(j) for j in ref["sel"])
    lam = dec["lam"].cpu().numpy()
    lam = lam[:, 0] + 1j * lam[:, 1]
    for j in ref["sel"]:
        want = ref["lam"][j]
        assert np.min(np.abs(lam[sel] - want)) < 1e-4 * abs(want), (j, want, lam[sel])
    bg = bg.cpu().numpy().T
    rel = np.linalg.norm(bg - ref_bg) / np.linalg.norm(ref_bg)
    assert rel <= 1e-3, rel
    got = C.unpack_mask(mask, clip.m)
    ref_mask = O.foreground_mask(Dm, ref_bg, tau)
    margin = np.abs(np.abs(Dm - ref_bg) - tau) > 0.5
    assert np.array_equal(got[margin], ref_mask[margin])
    f_gpu = O.fmeasure(got, clip.truth.T)[2]
    f_ref = O.fmeasure(ref_mask, clip.truth.T)[2]
    assert abs(f_gpu - f_ref) <= 1e-3, (f_gpu, f_ref)
    # the whole-pipeline entry point gives the same mask; it takes the
    # tensor-core subtract (mask only, BF16 hi + lo background), so decisions
    # within 0.01 grey of tau may differ from the CUDA-core pass above
    mask2 = C.cdmd_run_exact(ctx, D, C.make_params(1, r, K, tau, prec=prec))
    C.cdmd_status_sync(ctx)
    near = np.abs(np.abs(Dm - bg) - tau) <= 0.01
    assert near.mean() < 1e-3
    assert np.array_equal(C.unpack_mask(mask2, clip.m)[~near], got[~near])


def test_exact_dmd_rejects_bad_arguments(C, ctx):
    D = torch.zeros((300, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(C.CdmdError, match="UNSUPPORTED"):
        C.cdmd_snapshot_gram(ctx, D)                               # n > 256
    Du = torch.zeros((20, 4097), dtype=torch.uint8, device="cuda")[:, 1:]
    with pytest.raises(C.CdmdError, match="UNSUPPORTED"):
        C.cdmd_snapshot_gram(ctx, Du)                              # not 16-byte aligned
    R = torch.eye(20, dtype=torch.float64, device="cuda")
    with pytest.raises(C.CdmdError, match="INVALID_ARG"):
        C.cdmd_decompose_gram(ctx, R, 5, 3, selector="mlp")
    with pytest.raises(C.CdmdError, match="INVALID_ARG"):
        C.cdmd_decompose_gram(ctx, R, 20, 3)                       # r > n - 1
    with pytest.raises(C.CdmdError, match="INVALID_ARG"):
        C.cdmd_run_exact(ctx, D[:20], C.make_params(1, 5, 3, 25.0, selector="mlp"))
