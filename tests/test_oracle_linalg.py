"""Pins for the oracle's own SVD, eigen-solver and OMP (small inputs).

Each is checked against facts that do not come from the oracle: LAPACK via
numpy/scipy on small random matrices, reconstruction identities, and textbook
properties of orthogonal matching pursuit (exact for K = r, greedy top-K on an
orthonormal dictionary, never better than the best K-subset).
"""
import itertools

import numpy as np
import pytest

from oracle import cdmd as O


@pytest.mark.parametrize("shape", [(8, 8), (20, 8), (8, 20), (50, 19)])
def test_jacobi_svd_matches_lapack(shape):
    rng = np.random.default_rng(sum(shape))
    Y = rng.standard_normal(shape)
    U, s, V, sweeps = O.jacobi_svd(Y)
    s_ref = np.linalg.svd(Y, compute_uv=False)
    p = min(shape)
    np.testing.assert_allclose(s[:p], s_ref, rtol=1e-12, atol=1e-13 * s_ref[0])
    assert np.all(np.abs(s[p:]) < 1e-12 * s_ref[0])
    np.testing.assert_allclose(U[:, :p] * s[:p] @ V[:, :p].T, Y, atol=1e-12 * s_ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
    np.testing.assert_allclose(U[:, :p].T @ U[:, :p], np.eye(p), atol=1e-12)


def test_jacobi_svd_graded_singular_values():
    rng = np.random.default_rng(3)
    # orthonormal columns scaled over 11 decades: one-sided Jacobi keeps high
    # relative accuracy on column-scaled matrices (Demmel & Veselic, 1992)
    Qa, _ = np.linalg.qr(rng.standard_normal((30, 12)))
    sig = 10.0 ** -np.arange(12)
    Y = Qa * sig[None, :]
    _, s, _, _ = O.jacobi_svd(Y)
    np.testing.assert_allclose(s, sig, rtol=1e-12)


def test_hessenberg_form():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((9, 9))
    H, Q = O.hessenberg(A)
    assert np.all(np.abs(np.tril(H, -2)) == 0)
    np.testing.assert_allclose(Q @ Q.T, np.eye(9), atol=1e-13)
    np.testing.assert_allclose(Q @ H @ Q.T, A, atol=1e-12)


@pytest.mark.parametrize("n,seed", [(8, 0), (8, 1), (20, 2), (30, 3), (2, 4), (1, 5)])
def test_eig_matches_lapack(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    lam, W = O.eig_nonsymmetric(A)
    ref = np.linalg.eigvals(A)
    for x in ref:
        assert np.min(np.abs(lam - x)) < 1e-11 * max(1.0, abs(x))
    assert np.linalg.norm(A @ W - W * lam[None, :]) < 1e-11 * np.linalg.norm(A) * n
    np.testing.assert_allclose(np.linalg.norm(W, axis=0), 1.0, atol=1e-13)
    # ordering: non-increasing modulus
    assert np.all(np.diff(np.abs(lam)) <= 1e-12)


def test_eig_rotation_block_and_scaling():
    # closed form: a scaled rotation has eigenvalues rho e^{+-i theta}
    rho, th = 0.97, 0.3
    A = rho * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    lam, W = O.eig_nonsymmetric(A)
    np.testing.assert_allclose(lam, [rho * np.exp(1j * th), rho * np.exp(-1j * th)], atol=1e-14)
    # largest-modulus entry of each eigenvector is real positive
    for j in range(2):
        p = np.argmax(np.abs(W[:, j]))
        assert abs(W[p, j].imag) < 1e-15 and W[p, j].real > 0


def test_eig_upper_triangular_and_diagonal():
    T = np.triu(np.arange(1.0, 17.0).reshape(4, 4))
    lam, W = O.eig_nonsymmetric(T)
    np.testing.assert_allclose(np.sort(lam.real), np.sort(np.diag(T)), atol=1e-12)
    np.testing.assert_allclose(lam.imag, 0.0, atol=1e-12)


def _dictionary(k, r, seed, orthonormal=False):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((k, r)) + 1j * rng.standard_normal((k, r))
    if orthonormal:
        Phi, _ = np.linalg.qr(Phi)
    return Phi


def test_omp_with_k_equal_r_is_least_squares():
    Phi = _dictionary(40, 8, 0)
    y = np.random.default_rng(1).standard_normal(40)
    lam = np.linspace(1, 0.5, 8) + 0j
    sel, beta = O.omp(Phi, y, 8, lam)
    assert sorted(sel.tolist()) == list(range(8))
    full = np.zeros(8, dtype=complex)
    full[sel] = beta
    ref = np.linalg.lstsq(Phi, y.astype(complex), rcond=None)[0]
    np.testing.assert_allclose(full, ref, rtol=1e-10, atol=1e-12)


def test_omp_orthonormal_dictionary_takes_top_projections():
    Phi = _dictionary(30, 10, 2, orthonormal=True)
    y = np.random.default_rng(3).standard_normal(30) + 0j
    lam = np.ones(10, dtype=complex)
    proj = Phi.conj().T @ y
    for K in (1, 3, 5):
        sel, beta = O.omp(Phi, y, K, lam)
        top = np.argsort(-np.abs(proj))[:K]
        assert sel.tolist() == top.tolist()
        np.testing.assert_allclose(beta, proj[sel], rtol=1e-12, atol=1e-12)


def test_omp_recovers_exact_sparse_code():
    Phi = _dictionary(60, 12, 4)
    beta_true = np.zeros(12, dtype=complex)
    beta_true[[2, 7, 9]] = [3.0 - 1j, -2.0, 1.5j]
    y = Phi @ beta_true
    sel, beta = O.omp(Phi, y, 5, np.ones(12, dtype=complex))
    assert sorted(sel.tolist()) == [2, 7, 9]          # stops once residual ~ 0
    full = np.zeros(12, dtype=complex)
    full[sel] = beta
    np.testing.assert_allclose(full, beta_true, atol=1e-10)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_omp_never_beats_best_subset(K):
    Phi = _dictionary(20, 7, 10 + K)
    y = np.random.default_rng(K).standard_normal(20) + 0j
    sel, beta = O.omp(Phi, y, K, np.ones(7, dtype=complex))
    res_omp = np.linalg.norm(y - Phi[:, sel] @ beta)
    best = min(np.linalg.norm(y - Phi[:, list(S)] @ np.linalg.lstsq(Phi[:, list(S)], y, rcond=None)[0])
               for S in itertools.combinations(range(7), K))
    assert res_omp >= best - 1e-12
    if K == 1:
        assert abs(res_omp - best) < 1e-12        # one greedy step is optimal for unit-norm atoms


def test_omp_conjugate_tie_prefers_positive_imaginary_part():
    # a real target and a conjugate pair of atoms correlate equally
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    Phi = np.stack([phi.conj(), phi], axis=1)
    lam = np.array([0.9 - 0.1j, 0.9 + 0.1j])
    y = (phi + phi.conj()).real
    sel, _ = O.omp(Phi, y, 1, lam)
    assert sel.tolist() == [1]
