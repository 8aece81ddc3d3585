"""GPU parity of the learned selector's kernels against the FP64 oracle
(oracle/selector.py): gradient (1e-4 relative), Adam step, batch inference
(FP32 and BF16 operand rounding), features from the decomposition's Gram
quantities, learned selection inside cdmd_decompose with its OMP fallback,
and the device clip renderer against the host generator."""
import numpy as np
import pytest

import videogen
from oracle import cdmd as O
from oracle import measurement as M
from oracle import selector as S

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


def _rand_model(seed, N=1500):
    rng = np.random.default_rng(seed)
    X = (rng.normal(size=(N, 4)) * [2.0, 1.0, 3.0, 0.3] + [-0.1, 0.5, -2.0, 0.4]).astype(np.float32)
    Y = (rng.uniform(size=N) < 0.35).astype(np.float32)
    mu = np.array([-0.1, 0.5, -2.0, 0.4]) + 0.05
    sd = np.array([2.0, 1.0, 3.0, 0.3]) * 1.1
    theta = S.init_params(seed)
    theta[S.HIDDEN * S.N_FEAT:S.HIDDEN * S.N_FEAT + S.HIDDEN] = rng.normal(size=S.HIDDEN) * 0.3
    theta[-1] = 0.1
    blob = S.blob(theta, mu, sd, 0.05)
    return blob, X, Y


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("seed,N", [(0, 1), (1, 37), (2, 1500), (3, 100_003)])
def test_gradient_matches_oracle(C, ctx, seed, N):
    blob, X, Y = _rand_model(seed, N)
    loss, grad = C.cdmd_mlp_grad(ctx, _dev(blob), _dev(X), _dev(Y))
    C.cdmd_status_sync(ctx)
    theta, mu, sd, _ = S.from_blob(blob)
    l_ref, g_ref = S.loss_and_grad(theta, X, Y, mu, sd)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale
    big = np.abs(g_ref) > 1e-2 * scale
    assert np.max(np.abs(g[big] - g_ref[big]) / np.abs(g_ref[big])) <= 1e-4


def test_gradient_is_deterministic(C, ctx):
    blob, X, Y = _rand_model(4, 50_000)
    a = C.cdmd_mlp_grad(ctx, _dev(blob), _dev(X), _dev(Y))[1]
    b = C.cdmd_mlp_grad(ctx, _dev(blob), _dev(X), _dev(Y))[1]
    assert torch.equal(a, b)


def test_adam_steps_match_oracle(C, ctx):
    blob, X, Y = _rand_model(5, 3000)
    d = _dev(blob)
    m = torch.zeros(C.MLP_PARAMS, device="cuda")
    v = torch.zeros(C.MLP_PARAMS, device="cuda")
    theta, mu, sd, _ = S.from_blob(blob)
    mo = np.zeros_like(theta)
    vo = np.zeros_like(theta)
    lr = 1e-3
    for step in (1, 2, 3):
        loss = torch.zeros(1, device="cuda")
        C.cdmd_mlp_train_step(ctx, d, m, v, step, lr, _dev(X), _dev(Y), loss=loss)
        C.cdmd_status_sync(ctx)
        # oracle step from the device's parameters before the step
        l_ref, g = S.loss_and_grad(theta, X, Y, mu, sd)
        assert abs(loss.item() - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
        theta_new, mo, vo = S.adam_step(theta, mo, vo, g, step, lr)
        got = S.from_blob(d.cpu().numpy())[0]
        sig = np.abs(g) > 1e-2 * np.max(np.abs(g))
        # where the gradient is well resolved the FP32 update equals the FP64 one
        assert np.max(np.abs(got[sig] - theta_new[sig])) <= 1e-6 + 1e-3 * lr
        # elsewhere each update stays within Adam's step bound (lr times
        # ||a / sqrt(b)|| of the bias-corrected weights, below 1.01 for step <= 3)
        assert np.max(np.abs(got - theta)) <= 1.01 * lr + 1e-7
        np.testing.assert_allclose(m.cpu().numpy()[sig], mo[sig], rtol=1e-4)
        theta = got.astype(np.float64)
        mo = m.cpu().numpy().astype(np.float64)
        vo = v.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_oracle(C, ctx, bf16):
    blob, X, _ = _rand_model(6, 20_000)
    s, p = C.cdmd_mlp_forward(ctx, _dev(blob), _dev(X), bf16=bf16)
    C.cdmd_status_sync(ctx)
    theta, mu, sd, _ = S.from_blob(blob)
    s_ref, p_ref = S.forward(theta, X, mu, sd, bf16=bf16)
    ds = np.abs(s.cpu().numpy() - s_ref)
    if not bf16:
        assert np.max(ds / (1.0 + np.abs(s_ref))) <= 1e-5
    else:
        # identical BF16 operands; a hidden activation that the FP32 and FP64
        # sums round to neighbouring BF16 values moves s by one BF16 ulp of
        # that unit's term, so most rows agree to FP32 accuracy
        assert np.median(ds / (1.0 + np.abs(s_ref))) <= 1e-5
        assert np.max(ds / (1.0 + np.abs(s_ref))) <= 1e-2
    assert np.max(np.abs(p.cpu().numpy() - p_ref)) <= (1e-6 if not bf16 else 5e-3)


def _decomposed(C, ctx, seed, W=160, H=120, n=80, k=240, r=14, K=6):
    clip = videogen.make_clip(W, H, n, seed=seed)
    D = torch.from_numpy(clip.frames).cuda()
    DY = C.cdmd_sketch(ctx, D, k, 1000 + seed)
    dec = C.cdmd_decompose(ctx, DY, r, K, with_phiy=True)
    C.cdmd_status_sync(ctx)
    lam = torch.view_as_complex(dec["lam"]).cpu().numpy()
    PhiY = torch.view_as_complex(dec["PhiY"]).cpu().numpy().T      # (k, r)
    y1 = DY[0].cpu().numpy()
    return clip, D, DY, dec, lam, PhiY, y1


@pytest.mark.parametrize("seed", [0, 1])
def test_features_match_oracle(C, ctx, seed):
    r, K = 14, 6
    _, _, _, dec, lam, PhiY, y1 = _decomposed(C, ctx, seed, r=r, K=K)
    feats, lab = C.cdmd_selector_features(ctx, dec["lam"], dec["sel"], r, K)
    C.cdmd_status_sync(ctx)
    want = S.features(lam, PhiY, y1)
    np.testing.assert_allclose(feats.cpu().numpy(), want, rtol=1e-5, atol=1e-5)
    sel = dec["sel"].cpu().numpy()
    np.testing.assert_array_equal(lab.cpu().numpy(), S.labels(r, sel[sel >= 0]))


def _correlation_blob(tol):
    W1 = np.zeros((S.HIDDEN, S.N_FEAT))
    W1[0, 3] = 1.0
    W1[1, 0] = 0.5
    w2 = np.zeros(S.HIDDEN)
    w2[0] = 1.0
    w2[1] = -0.25
    return S.blob(S.pack(W1, np.zeros(S.HIDDEN), w2, 0.0), np.zeros(4), np.ones(4), tol)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_learned_selection_matches_oracle(C, seed):
    r = 14
    ctx = C.Context(0)
    blob = _correlation_blob(np.inf)
    C.cdmd_selector_load(ctx, _dev(blob))
    clip, D, DY, dec_omp, lam, PhiY, y1 = _decomposed(C, ctx, seed, r=r, K=6)
    theta, mu, sd, tol = S.from_blob(blob)
    # a K whose K-th and (K+1)-th logits are well apart, so the pick set is
    # unique (conjugate pairs score nearly alike)
    s_ref = np.sort(S.select(theta, mu, sd, tol, lam, PhiY, y1, 1)["s"])[::-1]
    K = next(q for q in (6, 5, 7, 4, 8, 3, 9) if s_ref[q - 1] - s_ref[q] > 1e-3)
    dec = C.cdmd_decompose(ctx, DY, r, K, selector="mlp", with_phiy=True)
    C.cdmd_status_sync(ctx)
    assert C.cdmd_selector_fallbacks(ctx) == 0
    assert torch.equal(dec["lam"], dec_omp["lam"])
    ref = S.select(theta, mu, sd, tol, lam, PhiY, y1, K, bf16=True)
    sel = dec["sel"].cpu().numpy()
    assert set(sel.tolist()) == set(ref["sel"].tolist())
    beta = torch.view_as_complex(dec["beta"]).cpu().numpy()
    fit = PhiY[:, sel] @ beta[sel]
    fit_ref = PhiY[:, ref["sel"]] @ ref["beta"]
    assert np.linalg.norm(fit - fit_ref) <= 1e-8 * np.linalg.norm(fit_ref)


def test_fallback_reproduces_omp_exactly(C):
    r, K = 14, 6
    ctx = C.Context(0)
    C.cdmd_selector_load(ctx, _dev(_correlation_blob(-1.0)))   # reject every learned pick
    _, _, DY, dec_omp, _, _, _ = _decomposed(C, ctx, 5, r=r, K=K)
    for rep in range(3):
        dec = C.cdmd_decompose(ctx, DY, r, K, selector="mlp")
        C.cdmd_status_sync(ctx)
        for key in ("sel", "beta", "nsel", "lam"):
            assert torch.equal(dec[key], dec_omp[key]), key
    assert C.cdmd_selector_fallbacks(ctx, reset=True) == 3
    assert C.cdmd_selector_fallbacks(ctx) == 0


def test_mlp_selector_requires_a_model(C):
    ctx = C.Context(0)
    DY = torch.zeros((20, 30), dtype=torch.float64, device="cuda")
    with pytest.raises(C.CdmdError):
        C.cdmd_decompose(ctx, DY, 4, 2, selector="mlp")


def test_synth_clip_matches_host_generator(C, ctx):
    # no noise: the same scene as the host generator up to FP32 vs FP64
    # rounding of the plane waves and of object-boundary tests
    spec = videogen.clip_spec(200, 150, 40, seed=17, drift=0.1, noise_sigma=0.0)
    host = videogen.make_clip(200, 150, 40, seed=17, drift=0.1, noise_sigma=0.0).frames
    D = C.cdmd_synth_clip(ctx, spec, seed=17).cpu().numpy()
    diff = np.abs(D.astype(np.int32) - host.astype(np.int32))
    assert np.mean(diff == 0) >= 0.99
    assert np.mean(diff > 1) <= 1e-3
    # noise: zero mean, sigma 3
    spec_n = dict(spec, noise_sigma=3.0)
    Dn = C.cdmd_synth_clip(ctx, spec_n, seed=17).cpu().numpy().astype(np.float64)
    inner = (D > 10) & (D < 245)
    e = (Dn - D)[inner]
    assert abs(e.mean()) < 0.02 and abs(e.std() - 3.0) < 0.05


def test_relabel_matches_oracle_omp(C, ctx):
    # OMP against a second target on the same decomposition: its own first
    # frame reproduces the decomposition's picks, a clean background frame
    # gives the oracle's OMP picks for that target.
    r, K = 14, 6
    clip, D, DY, dec, lam, PhiY, y1 = _decomposed(C, ctx, 8, r=r, K=K)
    own = C.cdmd_selector_relabel(ctx, DY, dec, r, DY[0].contiguous(), K)
    C.cdmd_status_sync(ctx)
    assert torch.equal(own, dec["sel"])
    bg = videogen.make_clip(160, 120, 2, seed=8, n_objects=0, noise_sigma=0.0).frames
    yt = C.cdmd_sketch(ctx, torch.from_numpy(bg).cuda(), 240, 1000 + 8)[0].contiguous()
    sel = C.cdmd_selector_relabel(ctx, DY, dec, r, yt, K)
    C.cdmd_status_sync(ctx)
    osel, _ = O.omp(PhiY, yt.cpu().numpy(), K, lam)
    np.testing.assert_array_equal(sel.cpu().numpy()[:len(osel)], osel)


@pytest.mark.parametrize("seed", [6, 7])
def test_committed_model_selection_matches_oracle(C, seed):
    # the trained model inside cdmd_decompose picks what the oracle's
    # BF16-emulated network picks, wherever the K-th logit is unambiguous
    from paper_1512_04205_gb300 import selector as SEL
    blob, _ = SEL.load_model()
    r = 20
    ctx = C.Context(0)
    C.cdmd_selector_load(ctx, _dev(blob))
    _, _, DY, dec_omp, lam, PhiY, y1 = _decomposed(C, ctx, seed, W=320, H=240, n=100, k=400, r=r, K=10)
    theta, mu, sd, tol = S.from_blob(blob)
    s_ref = np.sort(S.select(theta, mu, sd, np.inf, lam, PhiY, y1, 1)["s"])[::-1]
    K = next(q for q in (10, 9, 11, 8, 12, 7, 13) if s_ref[q - 1] - s_ref[q] > 1e-2)
    dec = C.cdmd_decompose(ctx, DY, r, K, selector="mlp", with_phiy=True)
    C.cdmd_status_sync(ctx)
    ref = S.select(theta, mu, sd, tol, lam, PhiY, y1, K, bf16=True)
    assert C.cdmd_selector_fallbacks(ctx) == int(ref["fallback"])
    assert set(dec["sel"].cpu().numpy().tolist()) == set(ref["sel"].tolist())
