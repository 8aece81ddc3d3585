"""Write the FP64 oracle's results for the 1920x1080 x 200-frame workload.

Calls only the oracle (oracle/) and the seeded input generator (videogen/).
The output, cdmd_1080p_x200.json beside this script, holds what the GPU
parity test of the benchmarked forms compares against:

* the clip: videogen.make_clip(1920, 1080, 200, seed=2024, drift=0.1) (the
  precision workload: six plane waves, three rectangles, +-10 % illumination
  ramp, noise sigma 3), with per-frame pixel sums and a SHA-256 of the frames
  so that a test can tell whether its own render matches;
* the sketch D_Y = C D (Algorithm 1 step 3, Eq. YCX) with the Gaussian C of
  seed 0x5EED1080, k = 1000, in FP64 over all 2,073,600 pixels: five full rows
  and the singular values of Y = D_Y[:, 0:n-1];
* the decomposition at r = 20 (Algorithm 1 steps 4-7): sigma, lambda,
  G = V S^-1 W;
* the selection of K = 10 modes by OMP on the compressed modes (Remark 3,
  Eq. sparsecoding) and by the learned selector with the model shipped with
  the package (the oracle's FP64 network with BF16 operand rounding), each
  with its amplitudes;
* for each selection, the oracle's mask over the whole clip (Eq. DMDTerms,
  MODULUS background; Eq. thres, tau = 25) scored against the generator's
  truth: TP, FP, FN and the F-measure (Section 4), and the number of
  pixel-frames within 0.5 grey of the threshold;
* for each selection, the oracle's background at BG_SAMPLES seeded
  (pixel, frame) points (numpy PCG64 seed BG_SEED: pixels first, then
  frames), which a benchmark can compare with the GPU's background without
  running the oracle.

Run:  python tests/golden/make_fullsize_1080p.py [--workers 8]
(about a minute of pixel work per core-minute; ~1-2 minutes on 8 cores).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "cdmd_1080p_x200.json")
MODEL = os.path.join(ROOT, "paper_1512_04205_gb300", "selector_model.json")

WORKLOAD = dict(width=1920, height=1080, n=200, clip_seed=2024, drift=0.1,
                k=1000, c_seed=0x5EED1080, ctype="gaussian", r=20, K=10, tau=25.0)
DY_ROWS = [0, 1, 511, 998, 999]
CHUNK = 16384
BG_SEED = 7
BG_SAMPLES = 8192


def bg_sample_points(m, n):
    """The seeded (pixel, frame) points of the stored background samples."""
    rng = np.random.default_rng(BG_SEED)
    return rng.integers(0, m, BG_SAMPLES), rng.integers(0, n, BG_SAMPLES)


def _sketch_chunk(args):
    """C[:, j0:j1] D[j0:j1, :] in FP64 for one pixel range (k x n)."""
    from oracle import measurement as M
    seed, k, j0, block = args
    Cb = M.gaussian_block(seed, np.arange(k), np.arange(j0, j0 + block.shape[1]))
    return Cb @ block.T.astype(np.float64)


def oracle_sketch(frames, k, seed, workers):
    n, m = frames.shape
    tasks = [(seed, k, j0, np.ascontiguousarray(frames[:, j0:j0 + CHUNK])) for j0 in range(0, m, CHUNK)]
    DY = np.zeros((k, n))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        # imap keeps the chunk order, so the FP64 sum order is fixed
        for part in pool.imap(_sketch_chunk, tasks, chunksize=1):
            DY += part
    return DY


def oracle_mask_counts(frames, truth, G, sel, beta, lam, tau):
    """Oracle mask over the whole clip, scored against truth, pixel chunk by chunk."""
    from oracle import cdmd as O
    n, m = frames.shape
    tp = fp = fn = near = 0
    Gs = G[:, sel]
    for j0 in range(0, m, 1 << 16):
        x = frames[:, j0:j0 + (1 << 16)].T.astype(np.float64)          # (pixels, n)
        Phi = O.lift(x, Gs)                                              # X' G_sel
        bg = O.background(Phi, beta, lam[sel], n)
        pred = O.foreground_mask(x, bg, tau)
        t = truth[:, j0:j0 + (1 << 16)].T
        tp += int(np.sum(pred & t))
        fp += int(np.sum(pred & ~t))
        fn += int(np.sum(~pred & t))
        near += int(np.sum(np.abs(np.abs(x - bg) - tau) <= 0.5))
    p = tp / (tp + fp) if tp + fp else 0.0
    rc = tp / (tp + fn) if tp + fn else 0.0
    f = 2 * p * rc / (p + rc) if p + rc else 0.0
    return dict(tp=tp, fp=fp, fn=fn, F=f, near_threshold=near)


def oracle_bg_samples(frames, G, sel, beta, lam):
    """Oracle background (MODULUS, Eq. DMDTerms) at the seeded sample points."""
    from oracle import cdmd as O
    n, m = frames.shape
    J, T = bg_sample_points(m, n)
    x = frames[:, J].T.astype(np.float64)                 # (samples, n): pixel J[i]'s time series
    bg = O.background(O.lift(x, G[:, sel]), beta, lam[sel], n)
    return [float(f"{v:.13g}") for v in bg[np.arange(len(J)), T]]


def cplx(a):
    a = np.asarray(a, dtype=np.complex128)
    return np.stack([a.real, a.imag], axis=-1).tolist()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args(argv)

    import videogen
    from oracle import cdmd as O
    from oracle import selector as S

    w = WORKLOAD
    t0 = time.time()
    clip = videogen.make_clip(w["width"], w["height"], w["n"], seed=w["clip_seed"], drift=w["drift"])
    frames, truth = clip.frames, clip.truth
    print(f"clip {time.time() - t0:.1f} s", flush=True)

    DY = oracle_sketch(frames, w["k"], w["c_seed"], args.workers)
    print(f"sketch {time.time() - t0:.1f} s", flush=True)
    dec = O.decompose(DY, w["r"], w["K"])
    sv = O.jacobi_svd(DY[:, :-1])[1]
    print(f"decompose {time.time() - t0:.1f} s", flush=True)

    with open(MODEL) as f:
        theta, mu, sd, tol = S.from_blob(json.load(f)["blob"])
    mlp = S.select(theta, mu, sd, tol, dec["lam"], dec["PhiY"], DY[:, 0], w["K"], bf16=True)

    omp_counts = oracle_mask_counts(frames, truth, dec["G"], dec["sel"], dec["beta"], dec["lam"], w["tau"])
    mlp_counts = oracle_mask_counts(frames, truth, dec["G"], mlp["sel"], mlp["beta"], dec["lam"], w["tau"])
    print(f"masks {time.time() - t0:.1f} s  F omp {omp_counts['F']:.6f}  F mlp {mlp_counts['F']:.6f}", flush=True)

    out = dict(
        what="FP64 oracle results for the 1920x1080x200 precision workload (tests/golden/make_fullsize_1080p.py)",
        workload=w,
        generator="videogen.make_clip(width, height, n, seed=clip_seed, drift=drift)",
        frames_sha256=hashlib.sha256(frames.tobytes()).hexdigest(),
        frame_sums=frames.sum(axis=1, dtype=np.int64).tolist(),
        truth_count=int(truth.sum()),
        dy_rows=DY_ROWS,
        dy=DY[DY_ROWS].tolist(),
        y_singular_values=sv.tolist(),
        sigma=dec["sigma"].tolist(),
        lam=cplx(dec["lam"]),
        G=cplx(dec["G"]),
        omp=dict(sel=dec["sel"].tolist(), beta=cplx(dec["beta"]), **omp_counts,
                 bg_samples=oracle_bg_samples(frames, dec["G"], dec["sel"], dec["beta"], dec["lam"])),
        mlp=dict(sel=np.asarray(mlp["sel"]).tolist(), beta=cplx(mlp["beta"]), fallback=bool(mlp["fallback"]),
                 residual=float(mlp["residual"]), tol=float(tol), **mlp_counts,
                 bg_samples=oracle_bg_samples(frames, dec["G"], mlp["sel"], mlp["beta"], dec["lam"])),
        bg_sample_seed=BG_SEED, bg_sample_count=BG_SAMPLES,
        y1_norm=float(np.linalg.norm(DY[:, 0])),
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    print(f"wrote {OUT} ({os.path.getsize(OUT)} bytes) in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
