"""Pins for the learned-selector oracle (features, network, loss, Adam,
selection with OMP fallback), each against a fact outside the code under
test: central finite differences, closed forms, hand-built networks and
dictionaries, and the sparse-coding solver itself."""
import numpy as np
import pytest

from oracle import cdmd as O
from oracle import selector as S


def _data(seed, N=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, S.N_FEAT)) * [2.0, 1.0, 3.0, 0.3] + [-0.1, 0.5, -2.0, 0.4]
    Y = (rng.uniform(size=N) < 0.4).astype(np.float64)
    mu = rng.normal(size=S.N_FEAT) * 0.1
    sd = rng.uniform(0.5, 2.0, size=S.N_FEAT)
    theta = S.init_params(seed)
    theta[S.HIDDEN * S.N_FEAT:S.HIDDEN * S.N_FEAT + S.HIDDEN] = rng.normal(size=S.HIDDEN) * 0.3
    theta[-1] = 0.2
    return theta, X, Y, mu, sd


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    theta, X, Y, mu, sd = _data(seed)
    _, g = S.loss_and_grad(theta, X, Y, mu, sd)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (S.loss_and_grad(tp, X, Y, mu, sd)[0] - S.loss_and_grad(tm, X, Y, mu, sd)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))
    # and relatively, on the entries that matter
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(fd[big] - g[big]) / np.abs(g[big])) < 1e-6


def test_zero_network_loss_is_log2_and_bias_gradient_closed_form():
    _, X, Y, mu, sd = _data(3)
    theta = np.zeros(S.N_PARAM)
    loss, g = S.loss_and_grad(theta, X, Y, mu, sd)
    assert loss == pytest.approx(np.log(2.0), rel=1e-15)
    assert g[-1] == pytest.approx(np.mean(0.5 - Y), rel=1e-14)
    assert np.all(g[:-1] == 0.0)


def test_forward_hand_built_l1_network():
    # units u < 4 compute relu(xh_u), units 4..7 relu(-xh_u); w2 sums them,
    # so s = ||xh||_1 + b2.
    theta, X, _, mu, sd = _data(4)
    W1 = np.zeros((S.HIDDEN, S.N_FEAT))
    W1[:4] = np.eye(4)
    W1[4:8] = -np.eye(4)
    w2 = np.zeros(S.HIDDEN)
    w2[:8] = 1.0
    th = S.pack(W1, np.zeros(S.HIDDEN), w2, -0.25)
    s, p = S.forward(th, X, mu, sd)
    want = np.abs((X - mu) / sd).sum(axis=1) - 0.25
    np.testing.assert_allclose(s, want, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(p, 1.0 / (1.0 + np.exp(-want)), rtol=1e-14)


def test_adam_closed_forms():
    rng = np.random.default_rng(5)
    theta = rng.normal(size=S.N_PARAM)
    g = rng.normal(size=S.N_PARAM)
    lr, eps = 3e-3, 1e-8
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    # With a constant gradient the bias-corrected moments are g and g^2 at
    # every step, so every update is -lr g / (|g| + eps).
    th = theta.copy()
    for step in range(1, 51):
        new, m, v = S.adam_step(th, m, v, g, step, lr, eps=eps)
        np.testing.assert_allclose(new - th, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
        th = new


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -3.14159,
                     1e-30, 65504.0, 0.1, -2.0 ** -130])
    rng = np.random.default_rng(6)
    vals = np.concatenate([vals, rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, 1000)])
    want = torch.from_numpy(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(vals), want)
    assert S.bf16_round(1.0 + 2.0 ** -8) == 1.0           # tie to even (down)
    assert S.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie to even (up)


def _orthonormal_dictionary(k, r, seed):
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(k, r)) + 1j * rng.normal(size=(k, r))
    Q, _ = np.linalg.qr(Z)
    return Q


def test_features_closed_form_and_invariances():
    k, r = 40, 6
    Q = _orthonormal_dictionary(k, r, 7)
    a = np.array([3.0, -1.0 + 2j, 0.5j, 0.0, 2.0, 1.0 - 1j])
    y1 = Q @ a
    lam = np.array([0.5 * np.exp(1j * np.pi / 3), 0.5 * np.exp(-1j * np.pi / 3), 1.0, -0.9, 0.0, 1j])
    X = S.features(lam, Q, y1)
    np.testing.assert_allclose(X[:, 0], [np.log(0.5), np.log(0.5), 0.0, np.log(0.9), S.FLOOR, 0.0], atol=1e-14)
    np.testing.assert_allclose(X[:, 1], [np.pi / 3, np.pi / 3, 0.0, np.pi, 0.0, np.pi / 2], atol=1e-14)
    np.testing.assert_allclose(X[:, 2], 0.0, atol=1e-14)
    np.testing.assert_allclose(X[:, 3], np.abs(a) / np.linalg.norm(a), atol=1e-14)
    # scaling the measurement scales y1 and Phi_Y together: features unchanged
    np.testing.assert_allclose(S.features(lam, 7.5 * Q, 7.5 * y1), X, atol=1e-13)
    # a column twice as long: f2 = log 2 - log 2 = 0 for it, -log 2 for the rest
    Q2 = Q.copy()
    Q2[:, 2] *= 2.0
    X2 = S.features(lam, Q2, y1)
    want = np.full(r, -np.log(2.0))
    want[2] = 0.0
    np.testing.assert_allclose(X2[:, 2], want, atol=1e-14)


def _correlation_network():
    # s = relu(f3) with mu = 0, sd = 1: probability increases with |phi^H y1|/||phi||
    W1 = np.zeros((S.HIDDEN, S.N_FEAT))
    W1[0, 3] = 1.0
    w2 = np.zeros(S.HIDDEN)
    w2[0] = 1.0
    return S.pack(W1, np.zeros(S.HIDDEN), w2, 0.0), np.zeros(4), np.ones(4)


def test_selection_equals_omp_on_orthonormal_dictionary():
    # OMP on an orthonormal dictionary picks the K largest |phi_j^H y1|, and
    # so does a network that is increasing in the correlation feature.
    k, r, K = 50, 10, 4
    Q = _orthonormal_dictionary(k, r, 8)
    a = np.array([5.0, 0.1, -4.0, 2.5j, 0.3, 1.0, -0.2, 3.0 + 1j, 0.05, 0.7])
    y1 = Q @ a + 1e-3 * (np.random.default_rng(9).normal(size=k))
    lam = np.exp(1j * np.linspace(-1, 1, r)) * 0.95
    theta, mu, sd = _correlation_network()
    out = S.select(theta, mu, sd, np.inf, lam, Q, y1, K, bf16=False)
    osel, obeta = O.omp(Q, y1, K, lam)
    assert set(out["sel"].tolist()) == set(osel.tolist())
    assert not out["fallback"]
    # the amplitudes are the projections of y1 on the chosen columns
    np.testing.assert_allclose(out["beta"], Q[:, out["sel"]].conj().T @ y1, atol=1e-12)


def test_fallback_returns_omp_exactly():
    rng = np.random.default_rng(10)
    k, r, K = 30, 8, 3
    PhiY = rng.normal(size=(k, r)) + 1j * rng.normal(size=(k, r))
    y1 = rng.normal(size=k)
    lam = rng.normal(size=r) + 1j * rng.normal(size=r)
    theta, mu, sd = _correlation_network()
    out = S.select(theta, mu, sd, -1.0, lam, PhiY, y1, K)
    osel, obeta = O.omp(PhiY, y1, K, lam)
    assert out["fallback"]
    np.testing.assert_array_equal(out["sel"], osel)
    np.testing.assert_array_equal(out["beta"], obeta)


def test_adam_on_bce_learns_a_separable_rule():
    # the gradient and the optimiser together descend: a threshold on one
    # feature is learned to full accuracy from a fixed start.
    rng = np.random.default_rng(11)
    X = rng.normal(size=(300, S.N_FEAT))
    Y = (X[:, 3] > 0.2).astype(np.float64)
    mu, sd = X.mean(axis=0), X.std(axis=0)
    theta = S.init_params(12)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    loss0 = S.loss_and_grad(theta, X, Y, mu, sd)[0]
    for step in range(1, 401):
        loss, g = S.loss_and_grad(theta, X, Y, mu, sd)
        theta, m, v = S.adam_step(theta, m, v, g, step, 1e-2)
    _, p = S.forward(theta, X, mu, sd)
    assert loss < 0.25 * loss0
    assert np.mean((p > 0.5) == (Y > 0.5)) >= 0.97


def test_blob_round_trip():
    theta, _, _, mu, sd = _data(13)
    b = S.blob(theta, mu, sd, 0.05)
    assert b.dtype == np.float32 and b.size == S.HEADER + S.N_PARAM
    th2, mu2, sd2, tol2 = S.from_blob(b)
    np.testing.assert_allclose(th2, theta.astype(np.float32))
    np.testing.assert_allclose(mu2, mu.astype(np.float32))
    assert tol2 == pytest.approx(0.05)
