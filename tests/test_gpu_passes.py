"""GPU parity of each pass against the FP64 oracle, on identical inputs.

Every test feeds the CUDA pass and the oracle the same seeded input (for the
later passes: the oracle's own upstream result), so each pass is checked on
its own.  Sizes span several tiles and a ragged tail (pixels not a multiple
of 32, frames not a multiple of 32, rows not a multiple of 4 or 64).
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- measurement

@pytest.mark.parametrize("ctype", ["gaussian", "rademacher"])
def test_measurement_entries_match_oracle(C, ctx, ctype):
    # A video whose frame t has a single pixel j_t = 1 sketches to DY[:, t] = C[:, j_t].
    m, k = 5000, 203
    probes = np.array([0, 1, 31, 32, 777, 1023, 2047, 4095, 4999, 2500, 123, 3333])
    frames = np.zeros((len(probes), m), dtype=np.uint8)
    frames[np.arange(len(probes)), probes] = 1
    seed = 0xDEADBEEF12345
    DY = C.cdmd_sketch(ctx, _dev(frames), k, seed, ctype=ctype).cpu().numpy()
    ref_fn = M.gaussian_block if ctype == "gaussian" else M.rademacher_block
    ref = ref_fn(seed, np.arange(k), probes)          # (k, len(probes))
    if ctype == "rademacher":
        np.testing.assert_array_equal(DY.T, ref)      # raw Philox bits: bit-exact
    else:
        err = np.abs(DY.T - ref)
        assert np.all(err <= 2e-6 * (1.0 + np.abs(ref))), err.max()


def test_sparse_measurement_csc_matches_oracle(C, ctx):
    m, k, density, seed = 3001, 97, 0.02, 77
    meas = C.Measure(ctx, "sparse", m, k, seed, density)
    ref = M.sparse_block(seed, np.arange(k), np.arange(m), density)
    assert meas.nnz == int(np.count_nonzero(ref))
    col_ptr = meas.col_ptr.cpu().numpy()
    codes = meas.row_idx.cpu().numpy().view(np.uint32)
    dense = np.zeros((k, m))
    for j in range(m):
        for e in range(col_ptr[j], col_ptr[j + 1]):
            dense[codes[e] & 0x7FFFFFFF, j] = -1.0 if codes[e] >> 31 else 1.0
    np.testing.assert_array_equal(dense, ref)


def test_rowsample_indices_match_oracle(C, ctx):
    # the last case keeps Floyd's set in global memory (2^15 slots > 96 KB)
    for m, k, seed in [(8_294_400, 1000, 3), (50, 50, 1), (1000, 7, 9), (2, 1, 4), (20_000, 19_990, 8),
                       (300_000, 12_000, 5)]:
        meas = C.Measure(ctx, "rowsample", m, k, seed)
        np.testing.assert_array_equal(meas.rows.cpu().numpy(), M.rowsample_indices(seed, k, m))


def test_rowsample_build_is_graph_capturable(C, ctx):
    """The single-pixel build runs on the device with no host round trip, so
    it can be captured in a CUDA graph and replayed."""
    m, k, seed = 8_294_400, 1000, 3
    side = torch.cuda.Stream()
    rows = torch.full((k,), -1, dtype=torch.int64, device="cuda")
    st = C.cdmd_measure()
    st.ctype, st.k, st.m, st.seed, st.density = C.CTYPES["rowsample"], k, m, seed, 0.0
    st.rows = rows.data_ptr()
    with torch.cuda.stream(side):
        C._check(ctx.lib.cdmd_measure_build(ctx.handle, C.ctypes.byref(st), C._stream(side)))   # sizes the workspace
    side.synchronize()
    rows.fill_(-1)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        C._check(ctx.lib.cdmd_measure_build(ctx.handle, C.ctypes.byref(st), C._stream(side)))
    torch.cuda.synchronize()
    rows.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rows.cpu().numpy(), M.rowsample_indices(seed, k, m))


# --------------------------------------------------------------------- sketch

@pytest.mark.parametrize("w,h,n,k", [(160, 120, 100, 200), (97, 61, 37, 203), (40, 30, 2, 1), (33, 9, 300, 65)])
def test_sketch_fp32_gaussian(C, ctx, w, h, n, k):
    clip = videogen.make_clip(w, h, n, seed=w + n)
    seed = 1234 + k
    DY = C.cdmd_sketch(ctx, _dev(clip.frames), k, seed).cpu().numpy().T      # (k, n)
    ref = O.sketch(M.measurement_matrix("gaussian", seed, k, clip.m), clip.video_matrix())
    scale = np.sqrt(clip.m) * 255.0
    assert np.abs(DY - ref).max() <= 2e-6 * scale


def test_sketch_fp32_rademacher_is_exact(C, ctx):
    clip = videogen.make_clip(97, 61, 37, seed=5)
    DY = C.cdmd_sketch(ctx, _dev(clip.frames), 130, 99, ctype="rademacher").cpu().numpy().T
    ref = O.sketch(M.measurement_matrix("rademacher", 99, 130, clip.m), clip.video_matrix())
    np.testing.assert_array_equal(DY, ref)


def test_sketch_respects_row_stride(C, ctx):
    clip = videogen.make_clip(50, 20, 12, seed=8)
    padded = np.zeros((12, 1040), dtype=np.uint8)
    padded[:, :1000] = clip.frames
    padded[:, 1000:] = 255                       # must be ignored
    D = _dev(padded)[:, :1000]
    DY = C.cdmd_sketch(ctx, D, 64, 5).cpu().numpy().T
    ref = O.sketch(M.measurement_matrix("gaussian", 5, 64, 1000), clip.video_matrix())
    assert np.abs(DY - ref).max() <= 2e-6 * np.sqrt(1000) * 255


@pytest.mark.parametrize("ctype", ["sparse", "rowsample"])
def test_sketch_gather_is_exact(C, ctx, ctype):
    clip = videogen.make_clip(97, 61, 45, seed=3)
    k, seed, density = 120, 21, 0.01
    meas = C.Measure(ctx, ctype, clip.m, k, seed, density)
    DY = C.cdmd_sketch_gather(ctx, _dev(clip.frames), meas).cpu().numpy().T
    ref = O.sketch(M.measurement_matrix(ctype, seed, k, clip.m, density=density), clip.video_matrix())
    np.testing.assert_array_equal(DY, ref)


# ------------------------------------------------------------------ decompose

def _match_pairs(a, b):
    """Greedy nearest matching of eigenvalue arrays; returns index into a for each b."""
    used, idx = set(), []
    for x in b:
        d = np.abs(a - x)
        d[list(used)] = np.inf
        j = int(np.argmin(d))
        used.add(j)
        idx.append(j)
    return np.array(idx)


def _phase_aligned_err(x, ref):
    alpha = np.vdot(x, ref) / np.vdot(x, x)
    return np.linalg.norm(alpha * x - ref) / np.linalg.norm(ref)


def _decompose_case(clip_args, k, r, K, seed):
    clip = videogen.make_clip(*clip_args, seed=seed)
    Cm = M.measurement_matrix("gaussian", seed + 1, k, clip.m)
    DY = O.sketch(Cm, clip.video_matrix())
    return clip, DY, O.decompose(DY, r, K)


@pytest.mark.parametrize("clip_args,k,r,K", [((160, 120, 100), 200, 10, 10),
                                             ((64, 48, 60), 120, 12, 5),
                                             ((48, 40, 33), 80, 20, 7)])
def test_decompose_matches_oracle(C, ctx, clip_args, k, r, K):
    clip, DY, ref = _decompose_case(clip_args, k, r, K, seed=clip_args[2])
    out = C.cdmd_decompose(ctx, _dev(DY.T), r, K, with_phiy=True)
    C.cdmd_status_sync(ctx)
    sigma = out["sigma"].cpu().numpy()
    np.testing.assert_allclose(sigma, ref["sigma"], rtol=1e-9)
    lam = torch.view_as_complex(out["lam"]).cpu().numpy()
    assert np.max(np.abs(lam - ref["lam"]) / np.abs(ref["lam"])) < 1e-8
    G = torch.view_as_complex(out["G"]).cpu().numpy()            # (r, n-1)
    for c in range(r):
        assert _phase_aligned_err(G[c], ref["G"][:, c]) < 1e-7
    PhiY = torch.view_as_complex(out["PhiY"]).cpu().numpy()       # (r, k)
    for c in range(r):
        assert _phase_aligned_err(PhiY[c], ref["PhiY"][:, c]) < 1e-7
    sel = out["sel"].cpu().numpy()
    nsel = int(out["nsel"].cpu().numpy()[0])
    assert nsel == len(ref["sel"])
    assert sorted(sel[:nsel].tolist()) == sorted(ref["sel"].tolist())
    assert np.all(sel[nsel:] == -1)
    # amplitudes enter only through Phi_Y[:, sel] beta (invariant to mode scaling)
    beta = torch.view_as_complex(out["beta"]).cpu().numpy()
    y_gpu = PhiY.T[:, sel[:nsel]] @ beta[sel[:nsel]]
    y_ref = ref["PhiY"][:, ref["sel"]] @ ref["beta"]
    assert np.linalg.norm(y_gpu - y_ref) <= 1e-8 * np.linalg.norm(y_ref)
    off = np.setdiff1d(np.arange(r), sel[:nsel])
    assert np.all(beta[off] == 0)


def test_decompose_lstsq_selects_all(C, ctx):
    clip, DY, ref = _decompose_case((64, 48, 40), 100, 8, 8, seed=2)
    out = C.cdmd_decompose(ctx, _dev(DY.T), 8, 8, selector="lstsq", with_phiy=True)
    C.cdmd_status_sync(ctx)
    PhiY = torch.view_as_complex(out["PhiY"]).cpu().numpy().T
    beta = torch.view_as_complex(out["beta"]).cpu().numpy()
    y1 = DY[:, 0]
    ref_beta = np.linalg.lstsq(PhiY, y1.astype(complex), rcond=None)[0]
    np.testing.assert_allclose(beta, ref_beta, rtol=1e-7, atol=1e-9 * np.abs(ref_beta).max())


def test_decompose_flags_rank_deficiency(C, ctx):
    # a static video has a rank-1 sketch: sigma_2 = 0 must be reported
    frames = np.full((20, 500), 77, dtype=np.uint8)
    DY = O.sketch(M.measurement_matrix("gaussian", 1, 40, 500), frames.T.astype(float))
    C.cdmd_decompose(ctx, _dev(DY.T), 3, 2)
    with pytest.raises(C.CdmdError) as e:
        C.cdmd_status_sync(ctx)
    assert e.value.status == 5
    C.cdmd_status_sync(ctx)                       # status is cleared after reading


def test_decompose_flags_nonfinite(C, ctx):
    DY = np.ones((30, 12))
    DY[3, 4] = np.nan
    C.cdmd_decompose(ctx, _dev(DY.T), 3, 2)
    with pytest.raises(C.CdmdError) as e:
        C.cdmd_status_sync(ctx)
    assert e.value.status == 6


def test_invalid_arguments_are_rejected(C, ctx):
    D = _dev(np.zeros((10, 100), dtype=np.uint8))
    with pytest.raises(C.CdmdError):
        C.cdmd_sketch(ctx, D, 0, 1)                       # k = 0
    DY = torch.zeros((10, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(C.CdmdError):
        C.cdmd_decompose(ctx, DY, 10, 3)                  # r > n-1
    with pytest.raises(C.CdmdError):
        C.cdmd_decompose(ctx, DY, 3, 4)                   # K > r
    with pytest.raises(ValueError):
        C.cdmd_sketch(ctx, D.float(), 4, 1)


# ----------------------------------------------------------------------- lift

@pytest.mark.parametrize("w,h,n,r", [(160, 120, 100, 10), (97, 61, 37, 13), (33, 9, 300, 30)])
def test_lift_fp32(C, ctx, w, h, n, r):
    clip = videogen.make_clip(w, h, n, seed=n)
    rng = np.random.default_rng(n)
    G = (rng.standard_normal((n - 1, r)) + 1j * rng.standard_normal((n - 1, r))) * 1e-3
    Gt = _dev(np.stack([G.T.real, G.T.imag], axis=-1))
    cols = np.array([r - 1, -1, 0, 2 % r], dtype=np.int32)
    Phi = C.cdmd_lift(ctx, _dev(clip.frames), Gt, cols=_dev(cols)).cpu().numpy()
    Phi = Phi[..., 0] + 1j * Phi[..., 1]
    ref = O.lift(clip.video_matrix(), G)
    for q, s in enumerate(cols):
        if s < 0:
            assert np.all(Phi[:, q] == 0)
        else:
            assert np.linalg.norm(Phi[:, q] - ref[:, s]) <= 2e-6 * np.linalg.norm(ref[:, s])


# ------------------------------------------------------------------- subtract

def _subtract_inputs(seed=4, w=97, h=61, n=45, r=8, K=5):
    clip = videogen.make_clip(w, h, n, seed=seed)
    Cm = M.measurement_matrix("gaussian", seed, 150, clip.m)
    out = O.cdmd(clip.video_matrix(), Cm, r, K)
    return clip, out


@pytest.mark.parametrize("mode", ["modulus", "real", "static"])
def test_subtract_matches_oracle(C, ctx, mode):
    clip, out = _subtract_inputs()
    sel = out["sel"]
    r = len(out["lam"])
    beta_full = np.zeros(r, dtype=complex)
    beta_full[sel] = out["beta"]
    Phi_sel = out["Phi"][:, sel].astype(np.complex64)
    Phi_t = _dev(np.stack([Phi_sel.real, Phi_sel.imag], axis=-1))
    beta_t = _dev(np.stack([beta_full.real, beta_full.imag], axis=-1))
    lam_t = _dev(np.stack([out["lam"].real, out["lam"].imag], axis=-1))
    mask, bg = C.cdmd_subtract(ctx, _dev(clip.frames), Phi_t, beta_t, lam_t, 25.0,
                               cols=_dev(sel.astype(np.int32)), mode=mode, want_bg=True)
    C.cdmd_status_sync(ctx)
    D = clip.video_matrix()
    ref_bg = O.background(out["Phi"][:, sel], out["beta"], out["lam"][sel], clip.n, mode)
    bg = bg.cpu().numpy().T
    assert np.abs(bg - ref_bg).max() <= 1e-4 * np.abs(ref_bg).max()
    ref_mask = O.foreground_mask(D, ref_bg, 25.0)
    margin = np.abs(np.abs(D - ref_bg) - 25.0) > 0.5
    got = C.unpack_mask(mask, clip.m)
    assert np.array_equal(got[margin], ref_mask[margin])
    # padding bits of the last word of every frame stay clear
    words = mask.cpu().numpy().view(np.uint32)
    tail = clip.m % 32
    if tail:
        assert np.all(words[:, -1] >> np.uint32(tail) == 0)
    np.testing.assert_array_equal(words, O.pack_mask(got))


# ----------------------------------------------------- sketch, tensor cores

@pytest.mark.parametrize("w,h,n,k", [(160, 120, 100, 200), (97, 61, 37, 203), (64, 33, 256, 300),
                                     (48, 32, 300, 120), (40, 24, 257, 64),
                                     (256, 160, 37, 100), (384, 160, 255, 200),   # odd n, several K steps per CTA
                                     (300, 40, 16, 513)])
def test_sketch_bf16x2_gaussian(C, ctx, w, h, n, k):
    # BF16 hi+lo C (2^-16 relative per entry), fast MUFU Box-Muller, FP32
    # accumulation: DY within 1e-4 of sqrt(m) * 255 of the FP64 oracle.
    clip = videogen.make_clip(w, h, n, seed=w + 7 * n)
    m = clip.m
    ldd = (m + 15) // 16 * 16
    padded = np.full((n, ldd), 255, dtype=np.uint8)     # bytes past m must be ignored
    padded[:, :m] = clip.frames
    D = _dev(padded)[:, :m]
    seed = 4242 + k
    DY = C.cdmd_sketch(ctx, D, k, seed, prec="bf16x2").cpu().numpy().T
    C.cdmd_status_sync(ctx)
    ref = O.sketch(M.measurement_matrix("gaussian", seed, k, m), clip.video_matrix())
    err = np.abs(DY - ref).max()
    assert err <= 1e-4 * np.sqrt(m) * 255.0, err
    # and it is a sketch of the same C as the FP32 path, not merely close in norm
    DY32 = C.cdmd_sketch(ctx, D, k, seed, prec="fp32").cpu().numpy().T
    rel = np.linalg.norm(DY - DY32) / np.linalg.norm(DY32)
    assert rel < 2e-5, rel


def test_sketch_bf16x2_rejects_unaligned_stride(C, ctx):
    frames = np.zeros((8, 1001), dtype=np.uint8)
    with pytest.raises(C.CdmdError):
        C.cdmd_sketch(ctx, _dev(frames), 64, 1, prec="bf16x2")     # ldd = 1001 is not a multiple of 16


# ------------------------------------------------------- lift, tensor cores

@pytest.mark.parametrize("w,h,n,r,modes", [(160, 120, 100, 10, [9, -1, 0, 2]), (97, 61, 37, 13, list(range(13))),
                                           (33, 9, 256, 30, list(range(29, 9, -1))), (300, 40, 2, 1, [0]),
                                           (48, 20, 300, 12, list(range(12))), (40, 16, 511, 6, [5, 0, 3])])
def test_lift_bf16x2(C, ctx, w, h, n, r, modes):
    # G scaled by a power of two per mode and split into FP16 hi+lo (about
    # 2^-21 relative), pixels exact in FP16: each Phi column within 5e-5 of
    # the FP64 oracle in 2-norm (G of size 1e-7 exercises the scaling).
    # Clips past 256 frames are lifted in chunks of at most 255 frames, the
    # later chunks adding into Phi.
    clip = videogen.make_clip(w, h, n, seed=n + r)
    m = clip.m
    ldd = (m + 15) // 16 * 16
    padded = np.full((n, ldd), 255, dtype=np.uint8)
    padded[:, :m] = clip.frames
    rng = np.random.default_rng(n)
    G = (rng.standard_normal((n - 1, r)) + 1j * rng.standard_normal((n - 1, r))) * 1e-7
    Gt = _dev(np.stack([G.T.real, G.T.imag], axis=-1))
    cols = np.array(modes, dtype=np.int32)
    Phi = C.cdmd_lift(ctx, _dev(padded)[:, :m], Gt, cols=_dev(cols), prec="bf16x2").cpu().numpy()
    C.cdmd_status_sync(ctx)
    Phi = Phi[..., 0] + 1j * Phi[..., 1]
    ref = O.lift(clip.video_matrix(), G)
    for q, s in enumerate(cols):
        if s < 0:
            assert np.all(Phi[:, q] == 0)
        else:
            err = np.linalg.norm(Phi[:, q] - ref[:, s]) / np.linalg.norm(ref[:, s])
            assert err <= 5e-5, (q, s, err)


def _conjugate_structured_modes(m, seed):
    # real eigenvalues with real modes and amplitudes, conjugate pairs with
    # conjugate modes and amplitudes, and one complex mode without partner
    rng = np.random.default_rng(seed)
    th = [0.3, 0.7, 1.1]
    lam = np.array([0.99, 0.95 * np.exp(1j * th[0]), 0.95 * np.exp(-1j * th[0]), 0.9 * np.exp(1j * th[1]),
                    0.9 * np.exp(-1j * th[1]), 0.8 * np.exp(1j * th[2]), 0.7])
    Phi = np.zeros((m, 7), dtype=complex)
    beta = np.zeros(7, dtype=complex)
    Phi[:, 0] = rng.normal(size=m)
    Phi[:, 6] = rng.normal(size=m)
    beta[0], beta[6] = 60.0, -8.0
    for lead in (1, 3):
        Phi[:, lead] = rng.normal(size=m) + 1j * rng.normal(size=m)
        Phi[:, lead + 1] = Phi[:, lead].conj()
        beta[lead] = rng.normal() * 10 + 1j * rng.normal() * 10
        beta[lead + 1] = beta[lead].conjugate()
    Phi[:, 5] = rng.normal(size=m) + 1j * rng.normal(size=m)
    beta[5] = 5.0 - 3.0j
    return lam, Phi, beta


@pytest.mark.parametrize("mode", ["modulus", "real", "static"])
@pytest.mark.parametrize("cols,perturb", [([0, 1, 2, 3, 4, 6], False),     # conjugate-closed: real terms
                                          ([0, 1, 2, 5, 3, 4], False),     # a lone complex mode
                                          ([0, 2, 1, 6], True)])           # pair amplitudes not conjugate
@pytest.mark.parametrize("pad", [0, 31])          # ldd = m (plain loads) or 16-byte aligned rows (tensor loads)
def test_subtract_real_terms_and_complex_path(C, ctx, mode, cols, perturb, pad):
    W, H, n = 61, 37, 45
    m = W * H
    lam, Phi, beta = _conjugate_structured_modes(m, 31)
    if perturb:
        beta = beta.copy()
        beta[2] = beta[1].conjugate() * (1 + 1e-3)
    frames = np.random.default_rng(32).integers(0, 256, size=(n, m), dtype=np.uint8)
    if pad:
        padded = np.full((n, m + pad), 255, dtype=np.uint8)      # bytes past m must be ignored
        padded[:, :m] = frames
        Dv = _dev(padded)[:, :m]
    else:
        Dv = _dev(frames)
    cols = np.array(cols, dtype=np.int32)
    Phi_sel = Phi[:, cols].astype(np.complex64)
    mask, bg = C.cdmd_subtract(ctx, Dv, _dev(np.stack([Phi_sel.real, Phi_sel.imag], axis=-1)),
                               _dev(np.stack([beta.real, beta.imag], axis=-1)),
                               _dev(np.stack([lam.real, lam.imag], axis=-1)), 25.0,
                               cols=_dev(cols), mode=mode, want_bg=True)
    C.cdmd_status_sync(ctx)
    ref_bg = O.background(Phi_sel.astype(np.complex128), beta[cols], lam[cols], n, mode)
    bg = bg.cpu().numpy().T
    assert np.abs(bg - ref_bg).max() <= 2e-5 * np.abs(ref_bg).max()
    D = frames.T.astype(np.float64)
    margin = np.abs(np.abs(D - ref_bg) - 25.0) > 0.01
    assert np.array_equal(C.unpack_mask(mask, m)[margin], O.foreground_mask(D, ref_bg, 25.0)[margin])
    # the mask without a background output takes the same decisions
    mask2 = C.cdmd_subtract(ctx, Dv, _dev(np.stack([Phi_sel.real, Phi_sel.imag], axis=-1)),
                            _dev(np.stack([beta.real, beta.imag], axis=-1)),
                            _dev(np.stack([lam.real, lam.imag], axis=-1)), 25.0, cols=_dev(cols), mode=mode)
    C.cdmd_status_sync(ctx)
    assert np.array_equal(C.unpack_mask(mask2, m)[margin], O.foreground_mask(D, ref_bg, 25.0)[margin])
