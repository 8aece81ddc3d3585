"""Automatic target rank on the device (Remark 2: the optimal hard threshold
for singular values, which Section 4 uses for every batch) against the
oracle's gd_rank on the same sketch.

The device reads the singular values of Y off the tridiagonal form of Y^T Y
(Sturm-count multisection for the median, one count for the rank); the oracle
takes the Jacobi SVD of Y.  Both see the same DY (the device sketch, copied
back), so tau agrees to rounding, and the ranks agree whenever no singular
value lies within 1e-6 of tau."""
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


def _oracle_rank(DY, r_max):
    DYh = DY.cpu().numpy().T               # k x n
    k, n = DYh.shape
    _, sv, _, _ = O.jacobi_svd(DYh[:, :-1])
    r, tau = O.gd_rank(sv, (k, n - 1), r_max)
    return r, tau, np.sort(sv)[::-1][:min(k, n - 1)]


@pytest.mark.parametrize("W,H,n,k,seed", [(160, 120, 100, 200, 0), (160, 120, 100, 200, 3), (96, 64, 80, 150, 1),
                                          (64, 48, 60, 40, 2)])
def test_auto_rank_matches_oracle(C, ctx, W, H, n, k, seed):
    # (64, 48, 60, 40): k < n - 1, so only k singular values are non-zero
    clip = videogen.make_clip(W, H, n, seed=seed)
    D = torch.from_numpy(clip.frames).cuda()
    DY = C.cdmd_sketch(ctx, D, k, 11 + seed)
    r_max = min(32, k, n - 1)
    out, r, tau = C.cdmd_decompose_auto(ctx, DY, r_max, 10)
    C.cdmd_status_sync(ctx)
    r_o, tau_o, sv = _oracle_rank(DY, r_max)
    assert abs(tau - tau_o) <= 1e-9 * tau_o, (tau, tau_o)
    assert np.min(np.abs(sv - tau_o)) > 1e-6 * tau_o       # no decision at the edge
    assert r == r_o and 1 < r < r_max
    # the rest of the decomposition is cdmd_decompose at that rank
    ref = C.cdmd_decompose(ctx, DY, r, min(10, r))
    C.cdmd_status_sync(ctx)
    assert torch.equal(out["lam"][:r], ref["lam"]) and torch.equal(out["sigma"][:r], ref["sigma"])
    assert torch.equal(out["sel"][:min(10, r)], ref["sel"]) and torch.equal(out["beta"][:r], ref["beta"])


def test_auto_rank_noise_signal_and_clamp(C, ctx):
    g = torch.Generator(device="cuda").manual_seed(4)
    k, n = 300, 90
    noise = torch.randn((n, k), dtype=torch.float64, device="cuda", generator=g)
    _, r, _ = C.cdmd_decompose_auto(ctx, noise, 20, 5)
    assert r == 1                                            # nothing above the noise floor
    U = torch.linalg.qr(torch.randn((k, 3), dtype=torch.float64, device="cuda", generator=g))[0]
    V = torch.linalg.qr(torch.randn((n, 3), dtype=torch.float64, device="cuda", generator=g))[0]
    signal = (V * torch.tensor([900.0, 600.0, 400.0], dtype=torch.float64, device="cuda")) @ U.T
    _, r, _ = C.cdmd_decompose_auto(ctx, signal + noise, 20, 5)
    assert r == 3
    out, r, _ = C.cdmd_decompose_auto(ctx, signal + noise, 2, 2)
    assert r == 2
    out, r, _ = C.cdmd_decompose_auto(ctx, signal + noise, 20, 5)
    sel = out["sel"].cpu().numpy()
    assert np.all(sel[3:] == -1)                             # K capped at the rank
    C.cdmd_status_sync(ctx)


def test_run_with_automatic_rank_matches_oracle(C, ctx):
    clip = videogen.make_clip(160, 120, 100, seed=5)
    k, K, tau, cseed = 200, 6, 25.0, 77
    Cm = M.measurement_matrix("gaussian", cseed, k, clip.m)
    Dm = clip.video_matrix()
    ref = O.decompose_auto(O.sketch(Cm, Dm), 32, K)
    ref_bg = O.background(O.lift(Dm, ref["G"])[:, ref["sel"]], ref["beta"], ref["lam"][ref["sel"]], clip.n)
    D = torch.from_numpy(clip.frames).cuda()
    mask = C.cdmd_run(ctx, D, C.make_params(k, 0, K, tau, seed=cseed))
    C.cdmd_status_sync(ctx)
    got = C.unpack_mask(mask, clip.m)
    margin = np.abs(np.abs(Dm - ref_bg) - tau) > 0.5
    assert np.array_equal(got[margin], O.foreground_mask(Dm, ref_bg, tau)[margin])
    # the same as the step-by-step calls at the rank the device chose
    DY = C.cdmd_sketch(ctx, D, k, cseed)
    dec, r, _ = C.cdmd_decompose_auto(ctx, DY, 32, K)
    assert r == ref["rank"]
    Phi = C.cdmd_lift(ctx, D, dec["G"][:r], cols=dec["sel"], ncols=min(K, r))
    mask2 = C.cdmd_subtract(ctx, D, Phi, dec["beta"][:r], dec["lam"][:r], tau, cols=dec["sel"])
    C.cdmd_status_sync(ctx)
    assert torch.equal(mask, mask2)


def test_auto_rank_rejects_bad_arguments(C, ctx):
    DY = torch.zeros((20, 50), dtype=torch.float64, device="cuda")
    for r_max, K in [(0, 1), (20, 3), (5, 6)]:                # r_max < 1, r_max > n - 1, K > r_max
        with pytest.raises(C.CdmdError, match="INVALID_ARG"):
            C.cdmd_decompose_auto(ctx, DY, r_max, K)
    D = torch.zeros((20, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(C.CdmdError, match="INVALID_ARG"):
        C.cdmd_run(ctx, D, C.make_params(50, 0, 25, 25.0))    # K above the automatic bound min(32, k, n-1) = 19
