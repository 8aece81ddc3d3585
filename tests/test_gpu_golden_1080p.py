"""End-to-end parity of the benchmarked forms at full size against the FP64
oracle's results for the same input (tests/golden/cdmd_1080p_x200.json,
written by tests/golden/make_fullsize_1080p.py from oracle/ alone).

Workload: videogen.make_clip(1920, 1080, 200, seed=2024, drift=0.1),
Gaussian C (seed 0x5EED1080, k = 1000), r = 20, K = 10, tau = 25 grey
(Algorithm 1 steps 2-9 with Remark 3; Eq. DMDTerms, MODULUS; Eq. thres).
The clip runs through cdmd_run_shared beside four device-rendered clips
under the same C, as the benchmark step does, in both forms:

* plain: FP32 sketch and lift, OMP selection;
* headline: BF16 hi+lo sketch and lift on the tensor cores, learned selector.

Checked against the oracle (which starts from the same uint8 frames, so an
error that enters in the sketch and propagates is measured):
* eigenvalues, matched one to one, on modes at least 1e-3 from any other:
  1e-5 relative (plain), 1e-4 (headline);
* the selected set (as a set) and, for the learned form, no fallback;
* the background on 100,000 seeded pixels x all 200 frames:
  ||bg_gpu - bg_oracle||_F / ||bg_oracle||_F <= 1e-4 (plain), 1e-3
  (headline), with bg_oracle = |X'[J] G_sel diag(beta) lambda^t| from the
  oracle's G, beta, lambda;
* mask bits on those pixels wherever | |x - bg_oracle| - tau | is more than
  0.5 grey and more than the largest background error seen;
* the F-measure of the whole GPU mask against the generator's truth within
  0.001 of the oracle's.
Measured errors are printed beside the bounds.

A further test reads entries of the tensor-core Gaussian generator one by
one: a clip whose frame t is a single bright pixel j_t sketches to
DY[:, t] = C[:, j_t], which the BF16 hi + lo split holds to 2^-16 relative.
"""
import json
import os

import numpy as np
import pytest

import videogen
from oracle import cdmd as O
from oracle import measurement as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cdmd_1080p_x200.json")


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


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        g = json.load(f)
    cp = lambda a: np.array([complex(x, y) for x, y in a])      # noqa: E731
    g["lam_c"] = cp(g["lam"])
    g["G_c"] = np.array([[complex(x, y) for x, y in row] for row in g["G"]])    # (n-1, r)
    for f in ("omp", "mlp"):
        g[f]["beta_c"] = cp(g[f]["beta"])
    return g


@pytest.fixture(scope="module")
def clip(gold):
    w = gold["workload"]
    c = videogen.make_clip(w["width"], w["height"], w["n"], seed=w["clip_seed"], drift=w["drift"])
    sums = c.frames.sum(axis=1, dtype=np.int64)
    diff = int(np.abs(sums - np.array(gold["frame_sums"])).sum())
    print(f"\nclip render vs golden: frame-sum difference {diff} grey levels over {c.frames.size} pixels")
    # a different libm may round an occasional pixel differently; that moves
    # results far below every tolerance here, but a different clip must not pass
    assert diff <= 1e-7 * c.frames.size * 128
    return c


def _bg_oracle(frames_J, g, form):
    """Oracle background at the sampled pixels (rows: pixels, columns: frames)."""
    sel = np.array(g[form]["sel"])
    x = frames_J.T.astype(np.float64)                       # (|J|, n)
    return O.background(O.lift(x, g["G_c"][:, sel]), g[form]["beta_c"], g["lam_c"][sel], x.shape[1]), x


def _match(lam_gpu, lam_ref):
    idx = [int(np.argmin(np.abs(lam_gpu - x))) for x in lam_ref]
    assert len(set(idx)) == len(idx), "eigenvalues do not match one to one"
    rel = np.abs(lam_gpu[idx] - lam_ref) / np.abs(lam_ref)
    sep = np.array([np.min(np.abs(np.delete(lam_ref, i) - x)) >= 1e-3 for i, x in enumerate(lam_ref)])
    return rel, sep, idx


@pytest.mark.parametrize("prec,selector", [("fp32", "omp"), ("bf16x2", "mlp")])
def test_benchmarked_form_matches_oracle_at_1080p(C, ctx, gold, clip, prec, selector):
    from paper_1512_04205_gb300 import selector as SEL
    w = gold["workload"]
    m, n, k, r, K, tau = clip.m, clip.n, w["k"], w["r"], w["K"], w["tau"]
    D = torch.from_numpy(clip.frames).cuda()
    others = []
    for i in range(1, 5):
        sd = w["clip_seed"] + 1000 * i
        others.append(C.cdmd_synth_clip(ctx, videogen.clip_spec(w["width"], w["height"], n, sd, drift=w["drift"]),
                                        sd))
    if selector == "mlp":
        C.cdmd_selector_load(ctx, torch.from_numpy(SEL.load_model()[0]).cuda())
        C.cdmd_selector_fallbacks(ctx, reset=True)
    p = C.make_params(k, r, K, tau, seed=w["c_seed"], prec=prec, selector=selector)
    masks = C.cdmd_run_shared(ctx, others + [D], p)          # the golden clip last: the workspace shows it
    C.cdmd_status_sync(ctx)
    v = C.workspace_tensors(ctx, m, n, k, r, K)
    torch.cuda.synchronize()
    form = "omp" if selector == "omp" else "mlp"
    g = gold[form]

    # eigenvalues (Algorithm 1 step 7)
    lam = torch.view_as_complex(v["lam"]).cpu().numpy()
    rel, sep, idx = _match(lam, gold["lam_c"])
    lam_tol = 1e-5 if prec == "fp32" else 1e-4
    print(f"\n[{prec}/{selector}] eigenvalues: max rel err {rel.max():.2e} (all), {rel[sep].max():.2e} "
          f"({int(sep.sum())} separated modes, bound {lam_tol:g})")
    assert rel[sep].max() <= lam_tol

    # selection (Remark 3 / learned)
    sel = v["sel"].cpu().numpy()
    assert set(sel.tolist()) == {idx[s] for s in g["sel"]}, (sel, g["sel"], idx)
    if selector == "mlp":
        assert C.cdmd_selector_fallbacks(ctx) == int(g["fallback"])

    # background on 100,000 seeded pixels, all frames (Eq. DMDTerms)
    rng = np.random.default_rng(11)
    J = np.unique(rng.integers(0, m, 100_000))
    Jt = torch.from_numpy(J).cuda()
    beta = v["beta"]
    _, bg = C.cdmd_subtract(ctx, D, v["Phi"], beta, v["lam"], tau, cols=v["sel"], want_bg=True)
    bg_gpu = bg[:, Jt].cpu().numpy().T.astype(np.float64)              # (|J|, n)
    del bg
    bg_ref, x = _bg_oracle(clip.frames[:, J], gold, form)
    bg_rel = np.linalg.norm(bg_gpu - bg_ref) / np.linalg.norm(bg_ref)
    bg_max = np.abs(bg_gpu - bg_ref).max()
    bg_tol = 1e-4 if prec == "fp32" else 1e-3
    print(f"[{prec}/{selector}] background: rel Frobenius err {bg_rel:.2e} (bound {bg_tol:g}), "
          f"max abs err {bg_max:.3f} grey over {len(J)} pixels x {n} frames")
    assert bg_rel <= bg_tol

    # mask bits away from the threshold (Eq. thres)
    mask = C.unpack_mask(masks[-1], m)
    want = O.foreground_mask(x, bg_ref, tau)
    margin = max(0.5, float(bg_max))
    far = np.abs(np.abs(x - bg_ref) - tau) > margin
    bad = int(np.sum((mask[J] != want) & far))
    print(f"[{prec}/{selector}] mask: {bad} bits differ of {int(far.sum())} more than {margin:.3f} grey from tau")
    assert bad == 0

    # F-measure of the whole mask against the generator's truth (Section 4)
    _, _, F = O.fmeasure(mask, clip.truth.T)
    print(f"[{prec}/{selector}] F-measure {F:.6f}, oracle {g['F']:.6f}, diff {abs(F - g['F']):.2e} (bound 1e-3)")
    assert abs(F - g["F"]) <= 1e-3


def test_tensor_core_gaussian_entries_match_oracle(C, ctx):
    """Entry by entry read-out of the BF16X2 sketch's Gaussian generator: a
    frame holding one pixel j_t = 1 sketches to DY[:, t] = C_hi + C_lo at
    (:, j_t).  The split holds C to 2^-16 relative (lo is C - hi rounded to
    BF16); the generator's hardware log2, square root and sine/cosine add an
    absolute error of a few 1e-6 (radius <= 6.8 times ~2^-21 relative
    errors), bounded here by 8e-6."""
    m, k = 5008, 1000                          # row stride a multiple of 16 (tensor copies)
    probes = np.array([0, 1, 31, 32, 63, 64, 777, 1023, 2047, 2048, 4095, 4999, 5007, 2500, 123, 3333])
    frames = np.zeros((len(probes), m), dtype=np.uint8)
    frames[np.arange(len(probes)), probes] = 1
    seed = 0x5EED1080
    DY = C.cdmd_sketch(ctx, torch.from_numpy(frames).cuda(), k, seed, prec="bf16x2").cpu().numpy()
    ref = M.gaussian_block(seed, np.arange(k), probes)            # (k, probes)
    err = np.abs(DY.T - ref)
    rel = err / np.maximum(np.abs(ref), 1e-30)
    excess = err - 2.0 ** -16 * np.abs(ref)
    print(f"\ntensor-core generator: {ref.size} entries, max abs err {err.max():.2e}, median rel err "
          f"{np.median(rel):.2e}, max err beyond the 2^-16 split bound {excess.max():.2e} (bound 8e-6)")
    assert np.all(err <= 2.0 ** -16 * np.abs(ref) + 8e-6)
