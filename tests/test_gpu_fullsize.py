"""Parity at full size, in the launch configuration the benchmark times, on
sampled outputs the FP64 oracle computes one by one:

* 1920x1080 x 200 frames, k = 1000, r = 20, K = 10 (the benchmark workload),
  mixed and plain precision: rows of the sketch D_Y against C_i . D; the
  small solves on the GPU's D_Y against the oracle's; sampled pixels of Phi
  against X'[j] G; sampled pixels of the background against the sum of
  Phi beta lambda^t, and their mask bits wherever |fg - tau| > 0.5.
* 3840x2160 x 300 frames (the gather workload): sampled rows of the sparse
  (density 1/1000) and single-pixel sketches exactly, and the decomposition
  at r = 30 on them.

Clips are rendered on the device (cdmd_synth_clip) and read back only where
the oracle needs them."""
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


def _render(C, ctx, w, h, n, seed, **gen):
    spec = videogen.clip_spec(w, h, n, seed, **gen)
    return C.cdmd_synth_clip(ctx, spec, seed)


def _sketch_rows(seed, rows, Dhost_chunks, m):
    """Oracle D_Y rows: C_i . D accumulated over pixel chunks (FP64)."""
    out = None
    for j0, block in Dhost_chunks:
        Cb = M.gaussian_block(seed, rows, np.arange(j0, j0 + block.shape[1]))
        part = Cb @ block.T.astype(np.float64)          # (rows, n)
        out = part if out is None else out + part
    return out


@pytest.fixture(scope="module")
def hd(C, ctx):
    W, H, n, k, r, K = 1920, 1080, 200, 1000, 20, 10
    D = _render(C, ctx, W, H, n, 2024, drift=0.1)
    return dict(D=D, W=W, H=H, n=n, k=k, r=r, K=K, m=W * H, seed=0x5EED1080)


@pytest.mark.parametrize("prec", ["bf16x2", "fp32"])
def test_fullsize_1080p_passes_on_sampled_outputs(C, ctx, hd, prec):
    D, m, n, k, r, K, seed = hd["D"], hd["m"], hd["n"], hd["k"], hd["r"], hd["K"], hd["seed"]
    DY = C.cdmd_sketch(ctx, D, k, seed, prec=prec)
    dec = C.cdmd_decompose(ctx, DY, r, K, with_phiy=True)
    Phi = C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K, prec=prec)
    mask, bg = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], 25.0, cols=dec["sel"], want_bg=True)
    C.cdmd_status_sync(ctx)

    # (a) sketch rows: C_i . D over all 2,073,600 pixels
    rows = np.array([0, 1, 511, 998, 999])
    chunk = 1 << 19
    chunks = [(j0, D[:, j0:j0 + chunk].cpu().numpy()) for j0 in range(0, m, chunk)]
    ref = _sketch_rows(seed, rows, chunks, m)
    got = DY.cpu().numpy().T[rows]
    err = np.abs(got - ref)
    if prec == "fp32":
        assert err.max() <= 1e-5 * np.sqrt(m) * 255.0
    else:
        # BF16 hi + lo C and FP32 accumulation in tensor memory: each CTA adds
        # its K steps (8 MMAs of 16 pixels each) into one FP32 partial, so a
        # partial carries at most n_acc ulps (2^-23 relative) of its size:
        # |err| <= n_acc 2^-23 |DY| when the partials add coherently.  Here
        # 32,400 K steps over 152 / 4 = 38 CTAs per row pair.
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        steps = (m + 63) // 64
        per_cta = -(-steps // max(1, sms // ((k + 255) // 256)))
        bound = per_cta * 8 * 2.0 ** -23
        scale = np.abs(ref).max()
        assert err.max() <= bound * scale, (err.max(axis=1).tolist(), scale, bound)

    # (b) small solves on the GPU's D_Y
    DYh = DY.cpu().numpy().T
    ref_dec = O.decompose(DYh, r, K)
    sig = dec["sigma"].cpu().numpy()
    np.testing.assert_allclose(sig, ref_dec["sigma"], rtol=1e-9)
    lam = torch.view_as_complex(dec["lam"]).cpu().numpy()
    idx = [int(np.argmin(np.abs(lam - x))) for x in ref_dec["lam"]]
    sep = np.array([np.min(np.abs(np.delete(ref_dec["lam"], i) - x)) >= 1e-3 for i, x in enumerate(ref_dec["lam"])])
    assert np.max((np.abs(lam[idx] - ref_dec["lam"]) / np.abs(ref_dec["lam"]))[sep]) < 1e-8

    # (c) lift on sampled pixels with the GPU's G: Phi[j] = X'[j, :] G[:, sel]
    rng = np.random.default_rng(5)
    J = np.unique(np.concatenate([rng.integers(0, m, 4000), [0, 1, m - 2, m - 1]]))
    Jt = torch.from_numpy(J).cuda()
    Xs = D[1:, Jt].cpu().numpy().T.astype(np.float64)                 # (|J|, n-1)
    G = torch.view_as_complex(dec["G"]).cpu().numpy().T                # (n-1, r)
    sel = dec["sel"].cpu().numpy()
    Phi_ref = Xs @ G[:, sel]
    Phi_got = torch.view_as_complex(Phi[Jt]).cpu().numpy()
    lift_tol = 5e-5 if prec == "bf16x2" else 1e-5
    assert np.abs(Phi_got - Phi_ref).max() <= lift_tol * np.abs(Phi_ref).max()

    # (d) background and mask on the sampled pixels with the GPU's Phi, beta, lambda
    beta = torch.view_as_complex(dec["beta"]).cpu().numpy()
    bg_ref = O.background(Phi_got.astype(np.complex128), beta[sel], lam[sel], n)   # (|J|, n)
    bg_got = bg[:, Jt].cpu().numpy().T
    assert np.abs(bg_got - bg_ref).max() <= 2e-5 * np.abs(bg_ref).max()
    x = D[:, Jt].cpu().numpy().T.astype(np.float64)
    want = O.foreground_mask(x, bg_ref, 25.0)
    bits = C.unpack_mask(mask, m)[J]
    margin = np.abs(np.abs(x - bg_ref) - 25.0) > 0.5
    assert np.array_equal(bits[margin], want[margin])


@pytest.fixture(scope="module")
def uhd(C, ctx):
    W, H, n = 3840, 2160, 300
    D = _render(C, ctx, W, H, n, 4321, n_objects=8, shape="ellipse")
    return dict(D=D, m=W * H, n=n)


def test_fullsize_4k_sparse_sketch_rows_exact(C, ctx, uhd):
    D, m, n = uhd["D"], uhd["m"], uhd["n"]
    k, seed, density = 1000, 77, 1e-3
    meas = C.Measure(ctx, "sparse", m, k, seed, density)
    DY = C.cdmd_sketch_gather(ctx, D, meas)
    C.cdmd_status_sync(ctx)
    got = DY.cpu().numpy().T
    for i in (0, 617):
        row = M.sparse_block(seed, [i], np.arange(m), density)[0]
        nz = np.nonzero(row)[0]
        Dz = D[:, torch.from_numpy(nz).cuda()].cpu().numpy().astype(np.float64)   # (n, nnz)
        np.testing.assert_array_equal(got[i], Dz @ row[nz])
    # the decomposition at r = 30 on the 4K gather sketch
    dec = C.cdmd_decompose(ctx, DY, 30, 10)
    C.cdmd_status_sync(ctx)
    ref = O.decompose(got, 30, 10)
    np.testing.assert_allclose(dec["sigma"].cpu().numpy(), ref["sigma"], rtol=1e-9)


def test_fullsize_4k_single_pixel_sketch_exact(C, ctx, uhd):
    D, m, n = uhd["D"], uhd["m"], uhd["n"]
    k, seed = 1000, 3
    meas = C.Measure(ctx, "rowsample", m, k, seed)
    DY = C.cdmd_sketch_gather(ctx, D, meas)
    C.cdmd_status_sync(ctx)
    rows = M.rowsample_indices(seed, k, m)
    ref = D[:, torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64).T
    np.testing.assert_array_equal(DY.cpu().numpy().T, ref)
