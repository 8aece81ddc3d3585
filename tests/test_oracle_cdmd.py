"""Method-level pins for the FP64 oracle (Algorithm 1, Remark 3, Eq. thres).

* C = I reduces compressed DMD to exact DMD: eigenvalues equal the non-zero
  eigenvalues of X' pinv_r(X), computed by brute force with LAPACK on the
  m x m matrix (Section 2.1 vs Section 3.2).
* A video that is exactly sum_j phi_j lambda_j^t (the DMD model, Eq. omegaj)
  returns its lambda_j to 1e-10 for any measurement with k >= r, and modes
  collinear with phi_j.
* Invariants: C Phi = Phi_Y; the background does not change when C is scaled
  or when eigenvectors are rescaled; eig(A~) equals the non-zero eigenvalues
  of Y' pinv_r(Y).
* Background modes, threshold mask and F-measure on hand-built cases.
"""
import numpy as np
import pytest

import videogen
from oracle import cdmd as O
from oracle import measurement as M


def _match(a, b):
    """Max distance from each entry of b to its nearest entry of a."""
    return max(np.min(np.abs(np.asarray(a) - x)) for x in np.asarray(b))


def _random_video(m, n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(m, n)).astype(np.float64)


@pytest.mark.parametrize("r", [19, 8])
def test_identity_measurement_is_exact_dmd(r):
    D = _random_video(64, 20, 0)                 # 8x8 frames, 20 frames
    X, Xp = O.split_snapshots(D)
    out = O.decompose(O.sketch(np.eye(64), D), r, K=r)
    # brute force: A_hat = X' pinv_r(X) on the 64 x 64 pixel space
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    pinv_r = Vt[:r].T @ np.diag(1.0 / s[:r]) @ U[:, :r].T
    ev = np.linalg.eigvals(Xp @ pinv_r)
    ev = ev[np.argsort(-np.abs(ev))][:r]
    scale = np.abs(ev).max()
    assert _match(out["lam"], ev) < 1e-10 * scale
    assert _match(ev, out["lam"]) < 1e-10 * scale


def _linear_dynamics_video(m, n, lam_half, seed):
    """Real video D = sum over conjugate pairs of phi lambda^t + conj."""
    rng = np.random.default_rng(seed)
    phis, lams = [], []
    for lam in lam_half:
        phi = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        phis += [phi, phi.conj()]
        lams += [lam, np.conj(lam)]
    Phi = np.stack(phis, axis=1)
    lams = np.array(lams)
    D = (Phi @ (lams[:, None] ** np.arange(n)[None, :])).real
    return D, Phi, lams


@pytest.mark.parametrize("ctype", ["gaussian", "rademacher", "sparse", "rowsample"])
def test_exact_linear_dynamics_recovered(ctype):
    lam_half = [0.999 * np.exp(0.05j), 0.95 * np.exp(0.4j), 0.9 * np.exp(1.1j)]
    m, n, r = 300, 30, 6
    D, Phi_true, lam_true = _linear_dynamics_video(m, n, lam_half, 1)
    k = 60
    C = M.measurement_matrix(ctype, 42, k, m, density=0.2)
    out = O.decompose(O.sketch(C, D), r, K=r)
    assert _match(out["lam"], lam_true) < 1e-10
    Phi = O.lift(D, out["G"])
    for j in range(r):
        i = int(np.argmin(np.abs(lam_true - out["lam"][j])))
        a, b = Phi[:, j], Phi_true[:, i]
        cos = abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 1 - 1e-10


def _small_clip_cdmd(K=4, scale=1.0, r=6, seed=3):
    clip = videogen.make_clip(32, 24, 24, seed=seed)
    D = clip.video_matrix()
    C = scale * M.measurement_matrix("gaussian", 5, 80, clip.m)
    return clip, D, C, O.cdmd(D, C, r, K)


def test_compressed_modes_are_sketched_full_modes():
    _, _, C, out = _small_clip_cdmd()
    np.testing.assert_allclose(C @ out["Phi"], out["PhiY"],
                               atol=1e-12 * np.abs(out["PhiY"]).max())


def test_atilde_eigenvalues_equal_projected_operator():
    _, _, _, out = _small_clip_cdmd()
    Y, Yp = out["DY"][:, :-1], out["DY"][:, 1:]
    r = len(out["lam"])
    U, s, Vt = np.linalg.svd(Y, full_matrices=False)
    pinv_r = Vt[:r].T @ np.diag(1.0 / s[:r]) @ U[:, :r].T
    ev = np.linalg.eigvals(Yp @ pinv_r)
    ev = ev[np.argsort(-np.abs(ev))][:r]
    assert _match(out["lam"], ev) < 1e-10 * np.abs(ev).max()


def _bg(out, D, mode=O.BG_MODULUS):
    sel = out["sel"]
    return O.background(out["Phi"][:, sel], out["beta"], out["lam"][sel], D.shape[1], mode)


def test_background_invariant_to_measurement_scale():
    clip, D, _, out1 = _small_clip_cdmd(scale=1.0)
    _, _, _, out2 = _small_clip_cdmd(scale=-3.7)
    np.testing.assert_allclose(_bg(out1, D), _bg(out2, D), rtol=1e-9, atol=1e-9)


def test_background_invariant_to_eigenvector_scaling():
    clip, D, C, out = _small_clip_cdmd()
    rng = np.random.default_rng(0)
    alpha = rng.standard_normal(len(out["lam"])) + 1j * rng.standard_normal(len(out["lam"]))
    G2 = out["G"] * alpha[None, :]
    PhiY2 = out["DY"][:, 1:] @ G2
    sel2, beta2 = O.omp(PhiY2, out["DY"][:, 0], 4, out["lam"])
    assert sorted(sel2.tolist()) == sorted(out["sel"].tolist())
    Phi2 = O.lift(D, G2)
    bg2 = O.background(Phi2[:, sel2], beta2, out["lam"][sel2], D.shape[1])
    np.testing.assert_allclose(bg2, _bg(out, D), rtol=1e-9, atol=1e-9)


def test_background_modes_static_real_modulus():
    clip, D, C, out = _small_clip_cdmd(K=6, r=6)      # all modes: real video
    bg_mod = _bg(out, D, O.BG_MODULUS)
    bg_re = _bg(out, D, O.BG_REAL)
    bg_st = _bg(out, D, O.BG_STATIC)
    # with every conjugate pair selected the reconstruction is real
    np.testing.assert_allclose(bg_mod, np.abs(bg_re), atol=1e-6 * bg_mod.max())
    np.testing.assert_allclose(bg_st, np.repeat(bg_mod[:, :1], D.shape[1], axis=1), atol=1e-9)
    # Eq. b as least squares: the residual of the all-mode fit of y1 is
    # orthogonal to every selected compressed mode (normal equations)
    y1 = out["DY"][:, 0]
    PhiS = out["PhiY"][:, out["sel"]]
    res = y1 - PhiS @ out["beta"]
    assert np.abs(PhiS.conj().T @ res).max() < 1e-9 * np.linalg.norm(PhiS, axis=0).max() * np.linalg.norm(y1)


def test_mask_threshold_is_strict():
    D = np.array([[100.0, 125.0, 126.0, 74.0, 75.0]])
    bg = np.full((1, 5), 100.0)
    mask = O.foreground_mask(D, bg, 25.0)
    assert mask.tolist() == [[False, False, True, True, False]]


def test_pack_mask_bit_layout():
    mask = np.zeros((70, 2), dtype=bool)
    mask[0, 1] = True
    mask[33, 1] = True
    mask[69, 0] = True
    words = O.pack_mask(mask)
    assert words.shape == (2, 3)
    assert words[1].tolist() == [1, 2, 0]
    assert words[0].tolist() == [0, 0, 1 << 5]


def test_fmeasure_hand_counts():
    pred = np.array([[1, 1, 0, 0], [1, 0, 0, 1], [0, 0, 0, 0], [0, 0, 0, 0]], dtype=bool)
    truth = np.array([[1, 1, 1, 0], [1, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]], dtype=bool)
    # TP = 3, FP = 1, FN = 1: P = 3/4, R = 3/4, F = 3/4
    p, r, f = O.fmeasure(pred, truth)
    assert (p, r) == (0.75, 0.75) and abs(f - 0.75) < 1e-15
    truth2 = truth.copy()
    truth2[3, 3] = True            # FN = 2: R = 3/5, F = 2*(3/4)(3/5)/(27/20) = 2/3
    p, r, f = O.fmeasure(pred, truth2)
    assert abs(r - 0.6) < 1e-15 and abs(f - 2.0 / 3.0) < 1e-15
    assert O.fmeasure(np.zeros((2, 2), bool), np.zeros((2, 2), bool)) == (0.0, 0.0, 0.0)


def test_generator_static_scene_and_truth():
    clip = videogen.make_clip(40, 30, 5, seed=9, n_objects=0, noise_sigma=0.0)
    assert not clip.truth.any()
    assert np.all(clip.frames == clip.frames[0:1])
    clip2 = videogen.make_clip(40, 30, 5, seed=9, n_objects=2, noise_sigma=0.0)
    # background pixels are untouched by the objects; object pixels are constant
    bgpix = ~clip2.truth
    np.testing.assert_array_equal(clip2.frames[bgpix], np.broadcast_to(clip.frames[0], clip.frames.shape)[bgpix])
    assert clip2.truth.any()
    clip3 = videogen.make_clip(40, 30, 9, seed=9, n_objects=0, noise_sigma=0.0, drift=0.1)
    mean = clip3.frames.astype(float).mean(axis=1)
    assert mean[-1] / mean[0] == pytest.approx(1.1 / 0.9, rel=0.02)
    # seeded: same seed, same clip
    again = videogen.make_clip(40, 30, 5, seed=9, n_objects=2)
    np.testing.assert_array_equal(again.frames, videogen.make_clip(40, 30, 5, seed=9, n_objects=2).frames)


def test_sharded_sketch_sums_to_full_sketch():
    # the sketch is linear in the pixels: per-shard sketches add up (used when
    # the pixel range is split between devices or thread blocks)
    clip = videogen.make_clip(32, 24, 12, seed=1)
    D = clip.video_matrix()
    C = M.measurement_matrix("gaussian", 2, 40, clip.m)
    full = O.sketch(C, D)
    bounds = [0, 100, 333, 500, clip.m]
    parts = sum(O.sketch(C[:, a:b], D[a:b]) for a, b in zip(bounds[:-1], bounds[1:]))
    np.testing.assert_allclose(parts, full, rtol=1e-12, atol=1e-9)


def test_exact_dmd_modes_are_eigenvectors_of_the_regression():
    # Section 2.1: A_hat = X' pinv(X); exact DMD's modes Phi = X' V S^-1 W
    # satisfy A_hat Phi = Phi Lambda (brute force on the 48 x 48 pixel space)
    D = _random_video(48, 30, 7)
    r = 12
    out = O.exact_dmd(D, r, K=4)
    X, Xp = O.split_snapshots(D)
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    pinv_r = Vt[:r].T @ np.diag(1.0 / s[:r]) @ U[:, :r].T
    A_hat = Xp @ pinv_r
    Phi, lam = out["Phi"], out["lam"]
    assert Phi.shape == (48, r)
    resid = np.linalg.norm(A_hat @ Phi - Phi * lam[None, :], axis=0) / np.linalg.norm(Phi, axis=0)
    assert resid.max() < 1e-9 * np.abs(lam).max()
    ev = np.linalg.eigvals(A_hat)
    ev = ev[np.argsort(-np.abs(ev))][:r]
    assert _match(lam, ev) < 1e-10 * np.abs(ev).max()
    # the selection picks K modes of Phi for x1 = D[:, 0] (Section 2.3)
    assert len(out["sel"]) == 4 and len(out["beta"]) == 4


def test_snapshot_gram_is_exact_and_matches_the_svd():
    rng = np.random.default_rng(2)
    D = rng.integers(0, 256, size=(500, 17), dtype=np.uint8)
    R = O.snapshot_gram(D)
    assert R.dtype == np.int64
    # brute force on a few entries, Python integers
    for s_, t_ in [(0, 0), (3, 11), (16, 2)]:
        assert R[s_, t_] == sum(int(D[j, s_]) * int(D[j, t_]) for j in range(500))
    assert np.array_equal(R, R.T)
    # eigenvalues of X^T X are the squared singular values of X, here from the
    # oracle's own Jacobi SVD (a different route from the Gram)
    X, _ = O.split_snapshots(D.astype(np.float64))
    _, sv, _, _ = O.jacobi_svd(X)
    ev = np.sort(np.linalg.eigvalsh(R[:-1, :-1].astype(np.float64)))[::-1]
    assert np.allclose(ev, np.sort(sv)[::-1] ** 2, rtol=1e-10, atol=1e-6 * ev[0])
