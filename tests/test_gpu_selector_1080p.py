"""The learned mode selector on held-out clips of the precision workload's
size (1920x1080, 200 frames, k = 1000, r = 20, K = 10; seeds never used in
training or calibration), against the sparse-coding selection it replaces
(Section 2.3, Eq. sparsecoding; Remark 3).

Per clip, on the GPU's BF16 hi+lo sketch: the decomposition with the learned
selector and with OMP, and the FP64 oracle's decomposition with OMP on the
same sketch.  Reported: the fallback count, whether the learned set equals
the oracle's OMP set, the background error of the learned form and of the
GPU's OMP form against the oracle's OMP background (20,000 seeded pixels x
all frames), and the F-measure of both GPU forms against the generator's
truth.  Asserted:
* the GPU's OMP form is within the mixed-precision bound (background 1e-3
  relative) of the oracle on every clip;
* where the learned set equals the oracle's, so is the learned form;
* on average the learned form's F-measure is no worse than OMP's by more
  than 0.01 (the selector is meant to pick background modes at least as
  well as sparse coding on the clip's own first frame).
"""
import numpy as np
import pytest

import videogen
from oracle import cdmd as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEEDS = [7_000_000 + i for i in range(10)]          # outside the training and calibration ranges
W, H, N, K_ROWS, R, K, TAU, C_SEED = 1920, 1080, 200, 1000, 20, 10, 25.0, 0x5EED1080


@pytest.fixture(scope="module")
def C():
    from paper_1512_04205_gb300 import build, cdmd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return cdmd


def _fmeasure(mask_words, truth, m):
    from paper_1512_04205_gb300 import cdmd as C
    pred = C.unpack_mask(mask_words, m)          # (m, n)
    t = truth.T
    tp = np.count_nonzero(pred & t)
    fp = np.count_nonzero(pred & ~t)
    fn = np.count_nonzero(~pred & t)
    p = tp / max(tp + fp, 1)
    rc = tp / max(tp + fn, 1)
    return 2 * p * rc / (p + rc) if p + rc > 0 else 0.0


def _form(C, ctx, D, dec, J):
    """Mask (device) and background at the sampled pixels (host, |J| x n) of
    one decomposition, lift and subtract on the tensor-core path."""
    Phi = C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K, prec="bf16x2")
    mask = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], TAU, cols=dec["sel"])
    _, bg = C.cdmd_subtract(ctx, D, Phi, dec["beta"], dec["lam"], TAU, cols=dec["sel"], want_bg=True)
    C.cdmd_status_sync(ctx)
    bgJ = bg[:, torch.from_numpy(J).cuda()].cpu().numpy().T.astype(np.float64)
    del bg
    return mask, bgJ


def test_learned_selector_on_held_out_1080p_clips(C):
    from paper_1512_04205_gb300 import selector as SEL
    ctx_mlp, ctx_omp = C.Context(0), C.Context(0)
    C.cdmd_selector_load(ctx_mlp, torch.from_numpy(SEL.load_model()[0]).cuda())
    C.cdmd_selector_fallbacks(ctx_mlp, reset=True)
    m = W * H
    J = np.unique(np.random.default_rng(12).integers(0, m, 20_000))
    rows = []
    for seed in SEEDS:
        spec = videogen.clip_spec(W, H, N, seed, drift=0.1)
        D = C.cdmd_synth_clip(ctx_omp, spec, seed)
        DY = C.cdmd_sketch(ctx_omp, D, K_ROWS, C_SEED, prec="bf16x2")
        dec_m = C.cdmd_decompose(ctx_mlp, DY, R, K, selector="mlp")
        dec_o = C.cdmd_decompose(ctx_omp, DY, R, K, selector="omp")
        C.cdmd_status_sync(ctx_mlp)
        C.cdmd_status_sync(ctx_omp)
        ref = O.decompose(DY.cpu().numpy().T, R, K)
        x = D[:, torch.from_numpy(J).cuda()].cpu().numpy().T.astype(np.float64)
        bg_ref = O.background(O.lift(x, ref["G"][:, ref["sel"]]), ref["beta"], ref["lam"][ref["sel"]], N)
        mask_m, bg_m = _form(C, ctx_mlp, D, dec_m, J)
        mask_o, bg_o = _form(C, ctx_omp, D, dec_o, J)
        truth = videogen.truth_from_spec(spec)
        lam_m = torch.view_as_complex(dec_m["lam"]).cpu().numpy()
        sel_m = {int(np.argmin(np.abs(ref["lam"] - lam_m[s]))) for s in dec_m["sel"].cpu().numpy() if s >= 0}
        rows.append(dict(seed=seed, same_set=sel_m == set(int(s) for s in ref["sel"]),
                         err_mlp=np.linalg.norm(bg_m - bg_ref) / np.linalg.norm(bg_ref),
                         err_omp=np.linalg.norm(bg_o - bg_ref) / np.linalg.norm(bg_ref),
                         F_mlp=_fmeasure(mask_m, truth, m), F_omp=_fmeasure(mask_o, truth, m)))
        del D
    fallbacks = C.cdmd_selector_fallbacks(ctx_mlp)
    print(f"\nlearned selector, {len(SEEDS)} held-out 1920x1080x200 clips: {fallbacks} fallbacks to OMP")
    for q in rows:
        print(f"  seed {q['seed']}: same set {q['same_set']!s:5s}  bg err vs oracle OMP: learned {q['err_mlp']:.2e}, "
              f"GPU OMP {q['err_omp']:.2e}  F: learned {q['F_mlp']:.4f}, OMP {q['F_omp']:.4f}")
    F_m = np.mean([q["F_mlp"] for q in rows])
    F_o = np.mean([q["F_omp"] for q in rows])
    print(f"  mean F: learned {F_m:.4f}, OMP {F_o:.4f}; identical sets on {sum(q['same_set'] for q in rows)} clips")
    assert all(q["err_omp"] <= 1e-3 for q in rows)
    assert all(q["err_mlp"] <= 1e-3 for q in rows if q["same_set"])
    assert F_m >= F_o - 0.01
