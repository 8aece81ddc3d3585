"""The small solves' FP64 reciprocal and reciprocal square root (Newton-Raphson
from the hardware approximations, two steps) against exact values.

Inputs sweep the normal FP64 range the solves can meet (2^-1000 .. 2^1000,
log-uniform, plus powers of two, their neighbours and mantissa extremes);
the exact 1/a and 1/sqrt(a) come from Python's decimal module at 50 digits,
and the error is measured in units in the last place of the exact value
(bound: 2 ulp).  The host's 1.0 / sqrt(a), which rounds twice, is printed
beside it as a yardstick.
"""
import decimal

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


def _inputs():
    rng = np.random.default_rng(2)
    a = [np.ldexp(1.0 + rng.random(20000), rng.integers(-1000, 1000, 20000))]
    e = np.arange(-1000, 1001, 37)
    p2 = np.ldexp(1.0, e)
    a += [p2, np.nextafter(p2, 0.0), np.nextafter(p2, np.inf), p2 * (2.0 - 2.0 ** -52), p2 * 1.5]
    a += [np.array([1.0, 2.0, 3.0, 0.1, 1e-300, 1e300, 7.0, 1.0 / 3.0])]
    return np.concatenate(a)


def _ulp_err(got, exact):
    """|got - exact| in ulps of the exact value (exact as Decimal)."""
    out = np.empty(len(got))
    for i, (g, x) in enumerate(zip(got, exact)):
        ulp = np.spacing(float(x))
        out[i] = float(abs(decimal.Decimal(float(g)) - x)) / ulp
    return out


def test_rcp64_rsqrt64_within_two_ulp(C):
    ctx = C.Context(0)
    a = _inputs()
    r, q = C.cdmd_selftest_recip(ctx, torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    r, q = r.cpu().numpy(), q.cpu().numpy()
    decimal.getcontext().prec = 50
    A = [decimal.Decimal(float(x)) for x in a]
    exact_r = [1 / x for x in A]
    exact_q = [1 / x.sqrt() for x in A]
    er = _ulp_err(r, exact_r)
    eq = _ulp_err(q, exact_q)
    ieee_q = 1.0 / np.sqrt(a)                      # two roundings: a yardstick, not the target
    print(f"\nrcp64: max {er.max():.3f} ulp, mean {er.mean():.3f}; rsqrt64: max {eq.max():.3f} ulp, mean "
          f"{eq.mean():.3f} (host 1/sqrt: max {_ulp_err(ieee_q, exact_q).max():.3f}) over {len(a)} inputs")
    assert np.all(np.isfinite(r)) and np.all(np.isfinite(q))
    assert er.max() <= 2.0
    assert eq.max() <= 2.0
