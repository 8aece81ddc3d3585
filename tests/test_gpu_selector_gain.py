"""What the trained selector gains over the plain method.

The committed model (paper_1512_04205_gb300/selector_model.json) was trained
on the GPU by the library's own kernels on 20,000 seeded 320x240x100 clips,
labelled by OMP against each clip's clean background frame.  On held-out
clips it is compared with the plain sparse-coding selection (OMP on the first
sketched frame, Remark 3 of the paper) through the same pipeline: F-measure
against the generator's ground-truth masks and background error against the
generator's object-free, noise-free background.  The fallback to OMP is
counted as well."""
import numpy as np
import pytest

import videogen
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


def _run(C, ctx, D, k, r, K, cseed, sel, tau=25.0):
    DY = C.cdmd_sketch(ctx, D, k, cseed)
    dec = C.cdmd_decompose(ctx, DY, r, K, selector=sel)
    Phi = C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K)
    mask, bg = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], tau, cols=dec["sel"], want_bg=True)
    C.cdmd_status_sync(ctx)
    return mask, bg.cpu().numpy().astype(np.float64)


def test_learned_selector_gain_on_held_out_clips(C):
    from paper_1512_04205_gb300 import selector as SEL
    blob, meta = SEL.load_model()
    ctx = C.Context(0)
    C.cdmd_selector_load(ctx, torch.from_numpy(blob).cuda())
    W, H, n, k, r, K, drift = 320, 240, 100, 400, 30, 10, 0.1
    seeds = range(7000, 7040)            # disjoint from the training seeds (>= 1,000,000)
    F = np.zeros((len(seeds), 2))
    E = np.zeros((len(seeds), 2))
    for q, s in enumerate(seeds):
        clip = videogen.make_clip(W, H, n, seed=s, drift=drift)
        bg_true = videogen.make_clip(W, H, n, seed=s, drift=drift, n_objects=0,
                                     noise_sigma=0.0).frames.astype(np.float64)
        D = torch.from_numpy(clip.frames).cuda()
        for c, sel in enumerate(("omp", "mlp")):
            mask, bg = _run(C, ctx, D, k, r, K, 77 + s, sel)
            F[q, c] = O.fmeasure(C.unpack_mask(mask, clip.m), clip.truth.T)[2]
            E[q, c] = np.linalg.norm(bg - bg_true) / np.linalg.norm(bg_true)
    fallbacks = C.cdmd_selector_fallbacks(ctx)
    gain_F = F[:, 1].mean() - F[:, 0].mean()
    gain_E = np.median(E[:, 0]) - np.median(E[:, 1])
    print(f"\nheld-out {len(seeds)} clips {W}x{H}x{n} r={r} K={K}: F omp {F[:, 0].mean():.4f} "
          f"learned {F[:, 1].mean():.4f} (gain {gain_F:+.4f}, better on {np.mean(F[:, 1] > F[:, 0]):.2f} of clips); "
          f"background error vs truth omp {np.median(E[:, 0]):.4f} learned {np.median(E[:, 1]):.4f}; "
          f"fallbacks {fallbacks}")
    assert fallbacks <= len(seeds) // 10
    assert gain_F > 0.0
    assert gain_E > 0.0
