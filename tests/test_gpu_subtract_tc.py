"""Pass (c) on the tensor cores (mask-only MODULUS / REAL calls with
32 <= n <= 1024 frames, taken 256 at most to a launch, up to 16 modes and a
16-byte aligned video) against
the FP64 oracle's background formula and threshold.

The background is a small GEMM in BF16 hi + lo with the three leading
products laid along K (about 2^-16 relative per term; the mode sums here stay
below a few hundred grey levels, so the error stays below 0.01 grey), so the
mask must equal the oracle's wherever |x - bg| sits more than 0.01 grey away
from tau, the same margin the CUDA-core pass meets; and it must equal the
CUDA-core pass's mask (taken with a background output, which stays on that
pass) there too.  Selections of real modes and complete conjugate pairs take
the real-sum form (one real term per pair, Re only); a lone complex mode
(r >= 5 here) takes the complex form."""
import numpy as np
import pytest

from oracle import cdmd as O

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _modes(m, r, seed):
    """r modes: conjugate pairs with conjugate modes and amplitudes, real
    modes, one unpaired complex mode; moduli from 0.9 to 1.01 (one mode
    grows over the clip), amplitudes that put the background near mid-grey."""
    rng = np.random.default_rng(seed)
    lam, Phi, beta = [], [], []
    while len(lam) < r:
        kind = len(lam) % 5
        if kind in (1, 3) and len(lam) + 2 <= r:
            z = rng.uniform(0.9, 1.01) * np.exp(1j * rng.uniform(0.05, 3.0))
            ph = rng.normal(size=m) + 1j * rng.normal(size=m)
            b = rng.normal() * 6 + 1j * rng.normal() * 6
            lam += [z, z.conjugate()]
            Phi += [ph, ph.conj()]
            beta += [b, b.conjugate()]
        elif kind == 4:
            lam.append(rng.uniform(0.9, 1.0) * np.exp(1j * rng.uniform(0.1, 2.0)))
            Phi.append(rng.normal(size=m) + 1j * rng.normal(size=m))
            beta.append(rng.normal() * 3 + 1j * rng.normal() * 3)
        else:
            lam.append(rng.uniform(0.95, 1.0))
            Phi.append(rng.normal(size=m) * 0.2 + 1.0)
            beta.append(120.0 if not lam[:-1] else rng.normal() * 8)
    return np.array(lam), np.stack(Phi, axis=1), np.array(beta)


# (W, H, n, r): a ragged pixel count (not a multiple of 32 or 128), the
# smallest n, odd n, the bench's n, the largest single launch, and clips
# past 256 frames (taken in frame chunks: 129 + 128, 150 + 150); 1 to 16 modes
CASES = [(61, 37, 32, 1), (61, 37, 45, 3), (97, 61, 200, 10), (128, 96, 256, 16), (40, 33, 111, 7),
         (300, 41, 64, 12), (64, 20, 257, 4), (160, 31, 300, 9)]


@pytest.mark.parametrize("mode", ["modulus", "real"])
@pytest.mark.parametrize("W,H,n,r", CASES)
def test_subtract_tc_matches_oracle(C, ctx, mode, W, H, n, r):
    m = W * H
    lam, Phi, beta = _modes(m, r, seed=W * 7 + n)
    frames = np.random.default_rng(n).integers(60, 200, size=(n, m), dtype=np.uint8)
    ldd = (m + 15) // 16 * 16
    padded = np.full((n, ldd), 255, dtype=np.uint8)       # bytes past m must be ignored
    padded[:, :m] = frames
    Dv = _dev(padded)[:, :m]
    cols = np.arange(r, dtype=np.int32)
    Phi_sel = Phi.astype(np.complex64)
    args = (Dv, _dev(np.stack([Phi_sel.real, Phi_sel.imag], axis=-1)), _dev(np.stack([beta.real, beta.imag], axis=-1)),
            _dev(np.stack([lam.real, lam.imag], axis=-1)), 25.0)
    mask = C.cdmd_subtract(ctx, *args, cols=_dev(cols), mode=mode)               # tensor-core pass
    mask_cc, _ = C.cdmd_subtract(ctx, *args, cols=_dev(cols), mode=mode, want_bg=True)   # CUDA-core pass
    C.cdmd_status_sync(ctx)
    ref_bg = O.background(Phi_sel.astype(np.complex128), beta, lam, n, mode)
    D = frames.T.astype(np.float64)
    margin = np.abs(np.abs(D - ref_bg) - 25.0) > 0.01
    assert margin.mean() > 0.99
    got = C.unpack_mask(mask, m)
    want = O.foreground_mask(D, ref_bg, 25.0)
    assert np.array_equal(got[margin], want[margin])
    assert np.array_equal(got[margin], C.unpack_mask(mask_cc, m)[margin])
    # a real mix of foreground and background decisions was exercised
    assert 0.01 < want.mean() < 0.99
    # bits past m in the last word of each frame stay clear
    words = mask.cpu().numpy().view(np.uint32)
    if m % 32:
        assert np.all(words[:, -1] >> np.uint32(m % 32) == 0)


def test_subtract_tc_selected_columns(C, ctx):
    # a selection list (cols) picks and orders modes; the pass must use the
    # amplitudes and powers of the selected columns only
    W, H, n, r = 96, 64, 120, 12
    m = W * H
    lam, Phi, beta = _modes(m, r, seed=5)
    cols = np.array([0, 3, 4, 1, 2, 9], dtype=np.int32)
    Phi_sel = Phi[:, cols].astype(np.complex64)
    frames = np.random.default_rng(6).integers(60, 200, size=(n, m), dtype=np.uint8)
    mask = C.cdmd_subtract(ctx, _dev(frames), _dev(np.stack([Phi_sel.real, Phi_sel.imag], axis=-1)),
                           _dev(np.stack([beta.real, beta.imag], axis=-1)),
                           _dev(np.stack([lam.real, lam.imag], axis=-1)), 25.0, cols=_dev(cols))
    C.cdmd_status_sync(ctx)
    ref_bg = O.background(Phi_sel.astype(np.complex128), beta[cols], lam[cols], n, "modulus")
    D = frames.T.astype(np.float64)
    margin = np.abs(np.abs(D - ref_bg) - 25.0) > 0.01
    assert np.array_equal(C.unpack_mask(mask, m)[margin], O.foreground_mask(D, ref_bg, 25.0)[margin])
