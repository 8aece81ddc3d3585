"""Pins of the oracle's SRFT measurement matrix C = R F D (Section 3.3,
"Measurement Matrices": subsampled randomized Fourier transform) against
facts outside it (CPU only):

* its real sketch rows are the real and imaginary parts of numpy's FFT of
  d * x at the kept frequencies (a library routine computing F);
* keeping every frequency (k = 2m) preserves energy: sum of squared sketch
  rows = m ||x||^2 (Parseval for the unnormalised DFT with |d_j| = 1);
* the kept frequencies are distinct, increasing and inside [0, m), and all
  of them are kept when ceil(k/2) = m;
* the diagonal's phases are uniform on the circle (mean of exp(i theta)
  near 0, mean of theta near pi).
"""
import numpy as np
import pytest

from oracle import measurement as M


@pytest.mark.parametrize("m,k,seed", [(60, 7, 3), (97, 40, 11), (128, 128, 5), (1920, 99, 2), (31, 62, 9)])
def test_srft_rows_are_fft_of_phased_frame(m, k, seed):
    C = M.measurement_matrix("srft", seed, k, m)
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, (m, 3)).astype(np.float64)
    freqs = M.srft_frequencies(seed, k, m)
    d = np.exp(1j * M.srft_phases(seed, np.arange(m)))
    Z = np.fft.fft(d[:, None] * x, axis=0)[freqs]               # (ceil(k/2), 3)
    Y = C @ x
    scale = np.abs(Z).max()
    assert np.max(np.abs(Y[0::2] - Z.real)) <= 1e-12 * scale * np.sqrt(m)
    assert np.max(np.abs(Y[1::2] - Z.imag[: Y[1::2].shape[0]])) <= 1e-12 * scale * np.sqrt(m)


def test_srft_all_frequencies_preserve_energy():
    m = 90
    C = M.measurement_matrix("srft", 4, 2 * m, m)
    x = np.random.default_rng(1).standard_normal(m)
    assert abs(np.sum((C @ x) ** 2) - m * np.sum(x ** 2)) <= 1e-10 * m * np.sum(x ** 2)


def test_srft_frequencies_distinct_sorted_in_range():
    for m, k, seed in [(1000, 61, 1), (50, 100, 2), (2_073_600, 1000, 3)]:
        f = M.srft_frequencies(seed, k, m)
        assert len(f) == (k + 1) // 2
        assert np.all(np.diff(f) > 0) and f[0] >= 0 and f[-1] < m
    assert np.array_equal(M.srft_frequencies(7, 100, 50), np.arange(50))


def test_srft_phases_uniform_on_circle():
    th = M.srft_phases(12, np.arange(200_000))
    assert np.all((th > 0) & (th < 2 * np.pi))
    assert abs(np.mean(np.exp(1j * th))) < 5.0 / np.sqrt(len(th))
    assert abs(np.mean(th) - np.pi) < 5.0 * (np.pi / np.sqrt(3)) / np.sqrt(len(th))
