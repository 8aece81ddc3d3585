"""Pins for the oracle's automatic target rank (Remark 2; Section 4's
evaluation settings): the optimal hard threshold for singular values of
Gavish and Donoho, tau = omega(beta) * median singular value.

* omega(beta): the oracle's published cubic approximation against the exact
  coefficient, computed here by another route: lambda*(beta) over the square
  root of the median of the Marchenko-Pastur law, the median found by
  numerical integration of the law's density.
* Hand-counted thresholds on short singular-value lists.
* Pure Gaussian noise keeps nothing (the rank clamps to 1); a rank-6 signal
  well above the noise floor plus noise keeps exactly 6.
* decompose_auto runs decompose at the chosen rank, with K capped by it.
"""
import numpy as np
import pytest

from oracle import cdmd as O


def _omega_exact(beta):
    integrate = pytest.importorskip("scipy.integrate")
    optimize = pytest.importorskip("scipy.optimize")
    lam_star = np.sqrt(2 * (beta + 1) + 8 * beta / ((beta + 1) + np.sqrt(beta ** 2 + 14 * beta + 1)))
    a, b = (1 - np.sqrt(beta)) ** 2, (1 + np.sqrt(beta)) ** 2

    def density(x):
        return np.sqrt(max((b - x) * (x - a), 0.0)) / (2 * np.pi * beta * x)

    def cdf(x):
        return integrate.quad(density, a, x, limit=200)[0]

    mu = optimize.brentq(lambda x: cdf(x) - 0.5, a, b)
    return lam_star / np.sqrt(mu)


@pytest.mark.parametrize("beta", [0.05, 0.2, 0.5, 0.75, 1.0])
def test_omega_cubic_matches_marchenko_pastur(beta):
    assert abs(O.gd_omega(beta) - _omega_exact(beta)) < 0.02


def test_omega_square_case_value():
    # beta = 1: lambda* = 4 / sqrt(3); the published coefficient is about 2.858
    assert abs(_omega_exact(1.0) - 2.858) < 2e-3


def test_threshold_hand_counts():
    # square, median 1: tau = omega(1) = 2.86 -> two values above
    r, tau = O.gd_rank([10.0, 9.0, 1.0, 1.0, 1.0], (5, 5), r_max=32)
    assert r == 2 and abs(tau - O.gd_omega(1.0)) < 1e-12
    # 2 x 6: only the two largest of six values count (min(shape) = 2),
    # median of (4, 2) = 3, beta = 1/3
    r, tau = O.gd_rank([4.0, 2.0, 0.0, 0.0, 0.0, 0.0], (2, 6), r_max=32)
    assert abs(tau - 3.0 * O.gd_omega(1 / 3)) < 1e-12 and r == 1
    # the clamp
    assert O.gd_rank([100.0] * 7 + [1.0] * 9, (16, 16), r_max=5)[0] == 5
    assert O.gd_rank([1.0] * 16, (16, 16), r_max=5)[0] == 1


def test_pure_noise_keeps_nothing_and_signal_keeps_its_rank():
    rng = np.random.default_rng(0)
    rows, cols = 1000, 199
    noise = rng.standard_normal((rows, cols))
    s = np.linalg.svd(noise, compute_uv=False)
    r, tau = O.gd_rank(s, (rows, cols), r_max=32)
    assert np.sum(s > tau) == 0 and r == 1
    U, _ = np.linalg.qr(rng.standard_normal((rows, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, 6)))
    strength = np.array([400.0, 300.0, 250.0, 200.0, 150.0, 120.0])
    s = np.linalg.svd(U @ np.diag(strength) @ V.T + noise, compute_uv=False)
    assert O.gd_rank(s, (rows, cols), r_max=32)[0] == 6


def test_decompose_auto_uses_the_threshold_rank():
    rng = np.random.default_rng(3)
    k, n = 120, 40
    t = np.arange(n)
    # three damped oscillations + a constant, plus noise: rank 7 in Y
    basis = [np.ones(n)] + [f(w * t) * 0.99 ** t for w in (0.3, 0.7, 1.3) for f in (np.cos, np.sin)]
    DY = sum(rng.standard_normal(k)[:, None] * b[None, :] * 50 for b in basis) + rng.standard_normal((k, n))
    out = O.decompose_auto(DY, r_max=20, K=10)
    _, sv, _, _ = O.jacobi_svd(DY[:, :-1])
    r, tau = O.gd_rank(sv, (k, n - 1), 20)
    assert out["rank"] == r == 7 and abs(out["rank_tau"] - tau) < 1e-12
    assert len(out["lam"]) == 7 and len(out["sel"]) == 7
