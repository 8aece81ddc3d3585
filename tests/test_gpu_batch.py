"""Batches of clips of uneven resolution and length (cdmd_batch_*): every clip
of a batch gets what a solo cdmd_run of the same clip gets, up to the
rounding order of the sketch's split sums, whether the batch runs eagerly,
as a captured graph, with grouped launches or with per-clip launches; graph
replays are bit-identical; the autotuner returns one of its candidates."""
import numpy as np
import pytest

import videogen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


# (width, height, n, k, r, K): uneven sizes, a clip longer than 256 frames,
# a pixel count that is not a multiple of the 960-pixel subtract tile
SHAPES = [(320, 240, 100, 400, 14, 8), (160, 120, 60, 240, 10, 6), (64, 48, 300, 300, 12, 10),
          (208, 96, 80, 320, 16, 10), (640, 480, 50, 200, 10, 4), (112, 80, 150, 600, 20, 10),
          (320, 192, 161, 644, 18, 10), (256, 128, 287, 1000, 27, 10)]     # odd n, several K steps per item


def _clips(device="cuda"):
    out = []
    for i, (w, h, n, k, r, K) in enumerate(SHAPES):
        clip = videogen.make_clip(w, h, n, seed=500 + i, drift=0.05)
        out.append(dict(D=torch.from_numpy(clip.frames).to(device), k=k, r=r, K=K, seed=9000 + i, clip=clip))
    return out


def _solo(C, ctx, c, prec, selector, tau=25.0):
    p = C.make_params(c["k"], c["r"], c["K"], tau, seed=c["seed"], prec=prec, selector=selector)
    mask = C.cdmd_run(ctx, c["D"], p)
    C.cdmd_status_sync(ctx)
    return mask


def _compare(C, batch, clips, ctx, prec, selector):
    for i, c in enumerate(clips):
        solo = _solo(C, ctx, c, prec, selector)
        got = batch.masks[i]
        m = c["D"].shape[1]
        a, b = C.unpack_mask(got, m), C.unpack_mask(solo, m)
        # the sketch sums split differently: decisions may move only at
        # pixels sitting on the threshold
        assert np.mean(a != b) <= 2e-4, (i, np.mean(a != b))
        v = batch.views(i)
        # the sketch matches the per-clip sketch up to the order of its FP32
        # partial sums: the batch may sum a clip's whole pixel range into one
        # partial (8 K16 products per 64-pixel step).  Accumulation in tensor
        # memory is not round-to-nearest: each add may lose up to an ulp of
        # the partial, the same way each time, so the error of a partial
        # grows with its length (terms x 2^-24 relative at worst); half that
        # bounds the difference between two partitions
        DYt = C.cdmd_sketch(ctx, c["D"], c["k"], c["seed"], prec=prec)
        DY = DYt.cpu().numpy()
        terms = 8 * -(-m // 64)
        assert np.abs(v["DY"] - DY).max() <= 5e-5 * np.abs(DY).max()
        assert np.linalg.norm(v["DY"] - DY) <= max(1e-5, 0.5 * terms * 2.0 ** -24) * np.linalg.norm(DY)
        # and so do the eigenvalues of the decomposition
        dec = C.cdmd_decompose(ctx, DYt, c["r"], c["K"], selector=selector)
        C.cdmd_status_sync(ctx)
        lam = torch.view_as_complex(dec["lam"]).cpu().numpy()
        idx = [int(np.argmin(np.abs(lam - x))) for x in v["lam"]]
        assert np.max(np.abs(lam[idx] - v["lam"]) / np.abs(v["lam"])) <= 1e-4


@pytest.mark.parametrize("prec,selector,grouped,graph", [("fp32", "omp", True, True), ("bf16x2", "omp", True, True),
                                                         ("bf16x2", "omp", False, True), ("fp32", "omp", True, False),
                                                         ("bf16x2", "lstsq", True, True)])
def test_batch_matches_solo_runs(C, prec, selector, grouped, graph):
    clips = _clips()
    batch = C.Batch(clips, 25.0, prec=prec, selector=selector, grouped=grouped, graph=graph, lanes=4)
    batch.run()
    batch.status_sync()
    ctx = C.Context(0)
    _compare(C, batch, clips, ctx, prec, selector)
    # replays are bit-identical
    first = [mk.clone() for mk in batch.masks]
    batch.run()
    batch.run()
    batch.status_sync()
    for a, b in zip(first, batch.masks):
        assert torch.equal(a, b)
    batch.close()


def test_batch_with_learned_selector(C):
    from paper_1512_04205_gb300 import selector as SEL
    blob = torch.from_numpy(SEL.load_model()[0]).cuda()
    clips = _clips()
    batch = C.Batch(clips, 25.0, prec="bf16x2", selector="mlp", selector_blob=blob, lanes=3)
    batch.run()
    batch.status_sync()
    ctx = C.Context(0)
    C.cdmd_selector_load(ctx, blob)
    _compare(C, batch, clips, ctx, "bf16x2", "mlp")
    batch.close()


def test_batch_autotune_picks_a_candidate(C):
    clips = _clips()
    batch = C.Batch(clips, 25.0, prec="bf16x2", autotune=True, lanes=8)
    t = batch.tuning()
    assert t["lanes"] in (2, 4, 8)
    assert t["waves"] in (1, 2, 4, 8)
    assert t["run_ms"] > 0.0
    assert t["sketch_steps"] >= 1 and t["subtract_tiles"] >= 1
    batch.run()
    batch.status_sync()
    ctx = C.Context(0)
    _compare(C, batch, clips, ctx, "bf16x2", "omp")
    batch.close()


def test_batch_rejects_a_bad_clip(C):
    clips = _clips()[:2]
    clips[1] = dict(clips[1], r=200)
    with pytest.raises(C.CdmdError, match="clip 1"):
        C.Batch(clips, 25.0)
