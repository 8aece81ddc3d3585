"""Failure detection without a GPU fault: a bounded wait that runs out.

cdmd_selftest_wait enqueues a kernel whose mbarrier nothing ever arrives at.
Its wait (the same bounded wait every tensor-core kernel uses) must give up
after its limit, report CDMD_ERR_TIMEOUT through cdmd_status_sync, and leave
the context usable: the next call on it computes the right result and reports
no error."""
import time

import numpy as np
import pytest

import videogen
from oracle import cdmd as O
from oracle import measurement as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


def test_bounded_wait_reports_timeout_and_context_recovers(C):
    ctx = C.Context(0)
    t0 = time.perf_counter()
    C.cdmd_selftest_wait(ctx, 50_000)                 # 50 ms
    with pytest.raises(C.CdmdError) as err:
        C.cdmd_status_sync(ctx)
    dt = time.perf_counter() - t0
    assert C.STATUS_NAMES[err.value.status] == "CDMD_ERR_TIMEOUT"
    assert 0.04 <= dt < 2.0, dt                       # gave up at its limit, not later
    # the status word was cleared and the context still works
    C.cdmd_status_sync(ctx)
    clip = videogen.make_clip(64, 48, 20, seed=4)
    DY = C.cdmd_sketch(ctx, torch.from_numpy(clip.frames).cuda(), 32, 7).cpu().numpy().T
    C.cdmd_status_sync(ctx)
    ref = O.sketch(M.measurement_matrix("gaussian", 7, 32, clip.m), clip.video_matrix())
    assert np.abs(DY - ref).max() <= 2e-6 * np.sqrt(clip.m) * 255.0


def test_timeout_stays_in_its_context(C):
    a, b = C.Context(0), C.Context(0)
    C.cdmd_selftest_wait(a, 20_000)
    with pytest.raises(C.CdmdError):
        C.cdmd_status_sync(a)
    C.cdmd_status_sync(b)                             # the other context saw nothing


def test_selftest_rejects_bad_limits(C):
    ctx = C.Context(0)
    for bad in (0, 2_000_001):
        with pytest.raises(C.CdmdError, match="limit_us"):
            C.cdmd_selftest_wait(ctx, bad)
