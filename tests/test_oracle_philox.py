"""Pins for the oracle's Philox4x32-10 and measurement-matrix draws.

Philox is pinned to an independent library implementation: cuRAND's host
generator CURAND_RNG_PSEUDO_PHILOX4_32_10 runs on the CPU and emits, for
output block q, Philox4x32-10 of counter (lo32(q>>16), hi32(q>>16), q&0xFFFF, 0)
under key (seed lo, seed hi).  Agreement over blocks that cross the 2^16
boundary and over offsets that reach counter word 1 exercises every key word
and counter words 0-2.  The draws built on top (Box-Muller normals,
+-1 signs, sparse entries, single-pixel rows) are pinned by their defining
distributions (Section 3.3 of the paper asks only for i.i.d. entries).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

from oracle import measurement as M
from oracle.philox import philox4x32_10, seed_key

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


def _curand_words(lib, seed, offset, count):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def _curand_counter(q):
    q = np.asarray(q, dtype=np.uint64)
    hi = q >> np.uint64(16)
    ctr = np.zeros(q.shape + (4,), dtype=np.uint32)
    ctr[..., 0] = (hi & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[..., 1] = (hi >> np.uint64(32)).astype(np.uint32)
    ctr[..., 2] = (q & np.uint64(0xFFFF)).astype(np.uint32)
    return ctr


@pytest.mark.parametrize("seed", [0x0123456789ABCDEF, 0xFEDCBA9876543210, 7])
def test_philox_matches_curand_host_stream(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    blocks = 65536 + 4096                         # crosses into counter word 0
    ref = _curand_words(lib, seed, 0, 4 * blocks)
    ours = philox4x32_10(_curand_counter(np.arange(blocks)), seed_key(seed)).reshape(-1)
    np.testing.assert_array_equal(ours, ref)


@pytest.mark.parametrize("q", [65536 * 3 + 7, 65536 * (1 << 32) + 5,
                               65536 * ((1 << 32) * 3 + 11) + 2,
                               65536 * ((1 << 32) * 0x3FF + 0x1234567) + 0xFFFF])
def test_philox_matches_curand_at_offsets(q):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    seed = 0x9E3779B97F4A7C15
    ref = _curand_words(lib, seed, 4 * q, 8)
    ours = philox4x32_10(_curand_counter(np.array([q, q + 1])), seed_key(seed)).reshape(-1)
    np.testing.assert_array_equal(ours, ref)


def test_philox_words_uniform_bytes():
    ctr = np.zeros((1 << 16, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(1 << 16)
    words = philox4x32_10(ctr, (3, 5))
    counts = np.bincount(words.view(np.uint8).reshape(-1), minlength=256)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4


def test_box_muller_closed_form_points():
    # U(w) = (w + 1/2) 2^-32.  With w_a = 2^31 the radius is sqrt(-2 ln U)
    # for U = 1/2 + 2^-33; w_b chosen at quarter turns gives cos/sin exactly.
    wa = np.array([2 ** 31], dtype=np.uint32)
    u_a = (2 ** 31 + 0.5) / 2 ** 32
    radius = np.sqrt(-2 * np.log(u_a))
    for wb, (cs, sn) in [(0, (1.0, 0.0)), (2 ** 30, (0.0, 1.0)),
                         (2 ** 31, (-1.0, 0.0)), (3 * 2 ** 30, (0.0, -1.0))]:
        z0, z1 = M.box_muller(wa, np.array([wb], dtype=np.uint32))
        assert abs(z0[0] - radius * cs) < 1e-8
        assert abs(z1[0] - radius * sn) < 1e-8


def test_gaussian_entries_are_standard_normal():
    C = M.gaussian_block(11, np.arange(64), np.arange(4096))
    z = C.reshape(-1)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair: radius^2 ~ chi^2_2, uncorrelated
    r2 = C[0::2, :] ** 2 + C[1::2, :] ** 2
    assert stats.kstest(r2.reshape(-1), "expon", args=(0, 2)).pvalue > 1e-3
    assert abs(np.corrcoef(C[0], C[1])[0, 1]) < 0.05
    # a row is a pure function of (seed, i, j): a sub-block equals the block
    sub = M.gaussian_block(11, np.array([5, 63]), np.array([17, 4095]))
    np.testing.assert_array_equal(sub, C[np.ix_([5, 63], [17, 4095])])


def test_rademacher_entries():
    C = M.rademacher_block(5, np.arange(256), np.arange(2048))
    assert set(np.unique(C)) == {-1.0, 1.0}
    assert abs(C.mean()) < 0.01
    # adjacent rows come from adjacent bits of one word: must be independent
    pairs = (C[0::2] > 0) * 2 + (C[1::2] > 0)
    counts = np.bincount(pairs.reshape(-1).astype(int), minlength=4)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_sparse_entries_density_and_signs():
    density = 1.0 / 50
    C = M.sparse_block(9, np.arange(400), np.arange(5000), density)
    nz = C != 0
    p_exact = M.sparse_threshold(density) / 2 ** 32
    expect = p_exact * C.size
    assert abs(nz.sum() - expect) < 5 * np.sqrt(expect)
    pos = (C > 0).sum()
    assert abs(pos - nz.sum() / 2) < 5 * np.sqrt(nz.sum() / 4)
    assert M.sparse_threshold(1e-3) == 4294967


def test_rowsample_distinct_sorted_uniform():
    idx = M.rowsample_indices(3, 1000, 8_294_400)
    assert len(idx) == 1000 and np.all(np.diff(idx) > 0)
    assert idx[0] >= 0 and idx[-1] < 8_294_400
    # every pixel is chosen with probability k/m
    m, k, trials = 40, 10, 4000
    hits = np.zeros(m)
    for s in range(trials):
        hits[M.rowsample_indices(s, k, m)] += 1
    assert stats.chisquare(hits).pvalue > 1e-4
    full = M.rowsample_indices(1, 16, 16)
    np.testing.assert_array_equal(full, np.arange(16))
