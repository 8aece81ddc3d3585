"""Measurement matrices C (k x m) of compressed DMD, FP64 oracle side.

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and
the benchmark's CPU-baseline leg may import it.

The paper (Section 3.3, "Measurement Matrices"; Algorithm 1 step 2) lists
dense i.i.d. Gaussian / sub-Gaussian (Bernoulli) matrices, very sparse random
projections with entries +1, 0, -1 of probabilities 1/(2s), 1-1/s, 1/(2s), and
single-pixel measurements (k rows of the identity drawn without replacement).
It does not say how the random numbers are drawn, so every entry here is a
pure function of (seed, row i, pixel j) through Philox4x32-10:

* Gaussian: counter (j, i//4, 0, 0); output word i%4.  Words (0,1) and (2,3)
  are Box-Muller pairs: with U(w) = (w + 1/2) 2^-32,
  z_even = sqrt(-2 ln U(w_a)) cos(2 pi U(w_b)),
  z_odd  = sqrt(-2 ln U(w_a)) sin(2 pi U(w_b)).
* Rademacher: counter (j, i//128, 1, 0); bit (i%128)%32 of word (i%128)//32;
  a clear bit is +1, a set bit is -1.
* Sparse (density 1/s): counter (j, i//4, 2, 0), word w = word i%4; the entry
  is non-zero iff w < floor(2^32 / s); then +1 if w is even, else -1.
* SRFT (subsampled randomized Fourier transform, C = R F D): D diagonal with
  entries d_j = exp(i theta_j) uniform on the complex unit circle,
  theta_j = 2 pi U(w0), w0 word 0 of counter (j, 0, 5, 0); F the unnormalised
  m-point DFT, F(f, j) = exp(-2 pi i f j / m); R keeps q = ceil(k/2) distinct
  frequencies s_0 < s_1 < ... drawn from [0, m) by Floyd's sampling on
  counters (t, 0, 6, 0) (as for the single-pixel rows).  The real sketch rows
  are the real and imaginary parts of those complex measurements:
  row 2a = Re(F D)[s_a, :] = cos(theta_j - 2 pi s_a j / m),
  row 2a+1 = Im(F D)[s_a, :] = sin(theta_j - 2 pi s_a j / m)
  (with odd k the last frequency keeps only its real row).
* Single pixel: Floyd's sampling of k distinct pixel indices in [0, m).  For
  t = m-k .. m-1 draw v uniform in [0, t] as the high 64 bits of
  (w1 * 2^32 + w0) * (t + 1), with (w0, w1) the first two words of counter
  (t, 0, 3, 0); insert v unless already taken, else insert t.  Rows of C are
  the selected pixels in increasing order.

Everything here is FP64 / exact integer arithmetic.
"""
import math

import numpy as np

from .philox import philox4x32_10, seed_key

STREAM_GAUSSIAN = 0
STREAM_RADEMACHER = 1
STREAM_SPARSE = 2
STREAM_ROWSAMPLE = 3
STREAM_SRFT_PHASE = 5
STREAM_SRFT_FREQ = 6

TWO_M32 = 2.0 ** -32


def uniform_open01(w):
    """Map uint32 words to (0, 1) as (w + 1/2) * 2^-32 (exact in FP64)."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * TWO_M32


def box_muller(wa, wb):
    """Two standard normals from two uint32 words (Box & Muller, 1958)."""
    u_a = uniform_open01(wa)
    u_b = uniform_open01(wb)
    radius = np.sqrt(-2.0 * np.log(u_a))
    angle = 2.0 * np.pi * u_b
    return radius * np.cos(angle), radius * np.sin(angle)


def gaussian_words_to_normals(words):
    """(..., 4) uint32 Philox output -> (..., 4) FP64 normals (lanes 0..3)."""
    z0, z1 = box_muller(words[..., 0], words[..., 1])
    z2, z3 = box_muller(words[..., 2], words[..., 3])
    return np.stack([z0, z1, z2, z3], axis=-1)


def gaussian_block(seed, rows, cols):
    """C[rows][:, cols] for the Gaussian measurement matrix, FP64.

    rows, cols: 1-D integer arrays of row indices i and pixel indices j.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    quads = np.unique(rows // 4)
    ctr = np.zeros((len(quads), len(cols), 4), dtype=np.uint32)
    ctr[..., 0] = cols[None, :]
    ctr[..., 1] = quads[:, None]
    ctr[..., 2] = STREAM_GAUSSIAN
    z = gaussian_words_to_normals(philox4x32_10(ctr, seed_key(seed)))
    qpos = np.searchsorted(quads, rows // 4)
    return z[qpos, :, rows % 4]


def rademacher_block(seed, rows, cols):
    """C[rows][:, cols] for the +-1 (Bernoulli) measurement matrix, FP64."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    groups = np.unique(rows // 128)
    ctr = np.zeros((len(groups), len(cols), 4), dtype=np.uint32)
    ctr[..., 0] = cols[None, :]
    ctr[..., 1] = groups[:, None]
    ctr[..., 2] = STREAM_RADEMACHER
    words = philox4x32_10(ctr, seed_key(seed)).astype(np.uint64)
    gpos = np.searchsorted(groups, rows // 128)
    b = rows % 128
    w = words[gpos, :, b // 32]                      # (len(rows), len(cols))
    bit = (w >> (b % 32).astype(np.uint64)[:, None]) & np.uint64(1)
    return np.where(bit == 0, 1.0, -1.0)


def sparse_threshold(density):
    """Integer acceptance threshold floor(2^32 * density) for a sparse entry."""
    return int(math.floor(4294967296.0 * float(density)))


def sparse_block(seed, rows, cols, density):
    """C[rows][:, cols] for the very sparse +-1/0 random projection, FP64."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    quads = np.unique(rows // 4)
    ctr = np.zeros((len(quads), len(cols), 4), dtype=np.uint32)
    ctr[..., 0] = cols[None, :]
    ctr[..., 1] = quads[:, None]
    ctr[..., 2] = STREAM_SPARSE
    words = philox4x32_10(ctr, seed_key(seed)).astype(np.int64)
    qpos = np.searchsorted(quads, rows // 4)
    w = words[qpos, :, rows % 4]
    thr = sparse_threshold(density)
    return np.where(w < thr, np.where(w % 2 == 0, 1.0, -1.0), 0.0)


def floyd_sample(seed, k, m, stream):
    """k distinct integers in [0, m), increasing: Floyd's algorithm with the
    step-t draw v = floor(((w1 << 32) | w0) (t + 1) / 2^64) from words 0, 1 of
    counter (t, 0, stream, 0)."""
    if not 0 < k <= m:
        raise ValueError("need 0 < k <= m")
    key = seed_key(seed)
    ts = np.arange(m - k, m, dtype=np.int64)
    ctr = np.zeros((k, 4), dtype=np.uint32)
    ctr[:, 0] = ts.astype(np.uint32)
    ctr[:, 2] = stream
    words = philox4x32_10(ctr, key)
    chosen = set()
    for t, w in zip(ts.tolist(), words.tolist()):
        u64 = (int(w[1]) << 32) | int(w[0])
        v = (u64 * (t + 1)) >> 64
        chosen.add(t if v in chosen else v)
    return np.array(sorted(chosen), dtype=np.int64)


def rowsample_indices(seed, k, m):
    """k distinct pixel indices in [0, m), increasing (Floyd's algorithm)."""
    return floyd_sample(seed, k, m, STREAM_ROWSAMPLE)


def srft_frequencies(seed, k, m):
    """The ceil(k/2) DFT rows R keeps, increasing (Floyd's algorithm)."""
    return floyd_sample(seed, (int(k) + 1) // 2, m, STREAM_SRFT_FREQ)


def srft_phases(seed, cols):
    """theta_j in [0, 2 pi) of the diagonal D for pixels cols (FP64)."""
    cols = np.asarray(cols, dtype=np.int64)
    ctr = np.zeros((len(cols), 4), dtype=np.uint32)
    ctr[:, 0] = cols.astype(np.uint32)
    ctr[:, 2] = STREAM_SRFT_PHASE
    w = philox4x32_10(ctr, seed_key(seed))[:, 0]
    return 2.0 * np.pi * uniform_open01(w)


def srft_block(seed, rows, cols, m, k):
    """C[rows][:, cols] of the real SRFT sketch (k rows, m pixels), FP64.

    The phase 2 pi s j / m is reduced exactly in integers (s j mod m, exact
    in int64 for m < 2^31) before the angle is formed."""
    if not 0 < m < 2 ** 31:
        raise ValueError("need 0 < m < 2^31")
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    freqs = srft_frequencies(seed, k, m)
    theta = srft_phases(seed, cols)
    s = freqs[rows // 2]
    red = (s[:, None] * cols[None, :]) % np.int64(m)
    ang = theta[None, :] - 2.0 * np.pi * red.astype(np.float64) / float(m)
    return np.where((rows % 2 == 0)[:, None], np.cos(ang), np.sin(ang))


def measurement_matrix(ctype, seed, k, m, density=None):
    """Dense FP64 C (k x m) for small sizes (tests)."""
    rows = np.arange(k)
    cols = np.arange(m)
    if ctype == "gaussian":
        return gaussian_block(seed, rows, cols)
    if ctype == "rademacher":
        return rademacher_block(seed, rows, cols)
    if ctype == "sparse":
        return sparse_block(seed, rows, cols, density)
    if ctype == "srft":
        return srft_block(seed, rows, cols, m, k)
    if ctype == "rowsample":
        c = np.zeros((k, m))
        c[np.arange(k), rowsample_indices(seed, k, m)] = 1.0
        return c
    if ctype == "identity":
        if k != m:
            raise ValueError("identity measurement needs k == m")
        return np.eye(m)
    raise ValueError(ctype)
