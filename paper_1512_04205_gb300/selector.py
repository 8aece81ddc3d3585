"""Training and evaluation driver of the learned background-mode selector.

Every arithmetic step runs in libcdmd's kernels: the clips are rendered on
the device (cdmd_synth_clip) from seeded scene parameters, sketched and
decomposed with the sparse-coding selection (OMP, Remark 3 of the paper),
their per-mode features and OMP labels exported (cdmd_selector_features),
and the network trained by cdmd_mlp_train_step (gradient + Adam kernels).
The host only draws scene parameters, shuffles row indices and keeps
counters.

    python -m paper_1512_04205_gb300.selector train --clips 20000 --out model.json
"""
import argparse
import json
import os
import time

import numpy as np

from . import cdmd as C

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "selector_model.json")

# training distribution: 320 x 240 clips of 100 frames, rank and drift drawn
# per clip, k = min(1000, 4 n), K = 10 background modes
TRAIN = dict(width=320, height=240, n=100, K=10, r_lo=10, r_hi=30, drift_hi=0.1)


def clip_setup(seed, width, height, n, r_lo, r_hi, drift_hi, **_):
    """Scene spec, rank and measurement seed of training clip `seed`."""
    import videogen
    rng = np.random.default_rng([seed, 0x5E1EC7])
    r = int(rng.integers(r_lo, r_hi + 1))
    drift = float(rng.uniform(0.0, drift_hi))
    spec = videogen.clip_spec(width, height, n, seed, drift=drift)
    return spec, r, int(rng.integers(1, 2**62))


def collect(device, clips, seed0, lanes=8, prec="fp32", cfg=TRAIN, with_residual=False, log_every=0,
            labels="clean"):
    """Features and OMP labels of `clips` seeded training clips.

    labels="clean": OMP picks against the sketch of the clip's clean
    background frame (frame 0 rendered without objects and noise, with the
    same measurement), which synthetic training data can supply and real
    video cannot; labels="y1": OMP picks against the clip's own first frame
    (the selection the decomposition makes at inference time).  Features are
    always those of the clip itself.

    Returns (X (rows x 4) float32 host array, Y (rows,) float32, meta) where
    meta lists, per clip, (seed, r, first row, OMP relative residual or nan).
    Clips are spread over `lanes` contexts and streams so that the small
    solves of several clips run at once."""
    import torch
    dev = torch.device("cuda", device)
    n, K = cfg["n"], cfg["K"]
    k = min(1000, 4 * n)
    ctxs = [C.Context(device) for _ in range(lanes)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(lanes)]
    feats, labs, meta = [], [], []
    pending = [None] * lanes
    t0 = time.time()

    skipped = []

    def drain(i):
        if pending[i] is None:
            return
        seed, r, f, y, res = pending[i]
        pending[i] = None
        try:
            C.cdmd_status_sync(ctxs[i], streams[i])
        except C.CdmdError as e:      # a numerical status: the clip is left out and reported
            skipped.append((seed, r, e.status))
            return
        feats.append(f.cpu().numpy())
        labs.append(y.cpu().numpy())
        meta.append((seed, r, res() if res is not None else float("nan")))

    for c in range(clips):
        i = c % lanes
        drain(i)
        seed = seed0 + c
        spec, r, cseed = clip_setup(seed, **cfg)
        with torch.cuda.stream(streams[i]):
            D = C.cdmd_synth_clip(ctxs[i], spec, seed)
            DY = C.cdmd_sketch(ctxs[i], D, k, cseed, prec=prec)
            dec = C.cdmd_decompose(ctxs[i], DY, r, K, selector="omp", with_phiy=with_residual)
            sel = dec["sel"]
            if labels == "clean":
                clean = dict(spec, n=2, objects=np.zeros((2, 0, 5)), noise_sigma=0.0)
                Dc = C.cdmd_synth_clip(ctxs[i], clean, seed)
                yt = C.cdmd_sketch(ctxs[i], Dc, k, cseed, prec=prec)[0]
                sel = C.cdmd_selector_relabel(ctxs[i], DY, dec, r, yt, K)
            f, y = C.cdmd_selector_features(ctxs[i], dec["lam"], sel, r, K)
        res = None
        if with_residual:
            res = _residual_fn(dec, DY)
        pending[i] = (seed, r, f, y, res)
        if log_every and (c + 1) % log_every == 0:
            print(f"collect {c + 1}/{clips} clips, {time.time() - t0:.1f} s", flush=True)
    for i in range(lanes):
        drain(i)
    rows = np.cumsum([0] + [f.shape[0] for f in feats])
    meta = [(s, r, int(rows[q]), res) for q, (s, r, res) in enumerate(meta)]
    if skipped:
        print(f"left out {len(skipped)} clips with a numerical status: {skipped[:20]}", flush=True)
    collect.skipped = skipped
    return np.concatenate(feats).astype(np.float32), np.concatenate(labs).astype(np.float32), meta


def _residual_fn(dec, DY):
    """Deferred host read of OMP's relative residual ||y1 - Phi_Y,S beta|| / ||y1||."""
    def f():
        PhiY = dec["PhiY"].cpu().numpy()
        PhiY = (PhiY[..., 0] + 1j * PhiY[..., 1]).T      # (k, r)
        beta = dec["beta"].cpu().numpy()
        beta = beta[:, 0] + 1j * beta[:, 1]
        y1 = DY[0].cpu().numpy()
        return float(np.linalg.norm(y1 - PhiY @ beta) / np.linalg.norm(y1))
    return f


def train(X, Y, device, epochs=30, batch=4096, lr=3e-3, seed=0, log=None):
    """Adam on the BCE loss with the device kernels; returns (blob, history)."""
    import torch
    dev = torch.device("cuda", device)
    rng = np.random.default_rng(seed)
    mu = X.mean(axis=0).astype(np.float64)
    sd = X.std(axis=0).astype(np.float64)
    sd = np.where(sd > 0, sd, 1.0)
    blob = np.zeros(C.MLP_BLOB, dtype=np.float32)
    blob[0:4] = mu
    blob[4:8] = sd
    blob[8] = np.inf
    W1 = rng.uniform(-1.0, 1.0, (C.MLP_HIDDEN, C.MLP_FEATURES)) * np.sqrt(6.0 / C.MLP_FEATURES)
    w2 = rng.uniform(-1.0, 1.0, C.MLP_HIDDEN) * np.sqrt(6.0 / C.MLP_HIDDEN) * 0.1
    o = C.MLP_HEADER
    blob[o:o + W1.size] = W1.ravel()
    blob[o + W1.size + C.MLP_HIDDEN:o + W1.size + 2 * C.MLP_HIDDEN] = w2
    ctx = C.Context(device)
    dblob = torch.from_numpy(blob).to(dev)
    m = torch.zeros(C.MLP_PARAMS, dtype=torch.float32, device=dev)
    v = torch.zeros(C.MLP_PARAMS, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    N = X.shape[0]
    step = 0
    history = []
    for ep in range(epochs):
        perm = rng.permutation(N)
        Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
        Yd = torch.from_numpy(np.ascontiguousarray(Y[perm])).to(dev)
        losses = []
        for b0 in range(0, N, batch):
            step += 1
            C.cdmd_mlp_train_step(ctx, dblob, m, v, step, lr, Xd[b0:b0 + batch], Yd[b0:b0 + batch], loss=loss)
            losses.append(loss.clone())
        ep_loss = float(torch.stack(losses).mean().item())
        history.append(ep_loss)
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {ep_loss:.5f}")
    C.cdmd_status_sync(ctx)
    return dblob.cpu().numpy(), history


def accuracy(blob, X, Y, device, bf16=True):
    """Fraction of rows whose thresholded probability matches the label."""
    import torch
    dev = torch.device("cuda", device)
    ctx = C.Context(device)
    _, p = C.cdmd_mlp_forward(ctx, torch.from_numpy(blob).to(dev), torch.from_numpy(X).to(dev), bf16=bf16)
    return float(((p.cpu().numpy() > 0.5) == (Y > 0.5)).mean())


def learned_residuals(device, blob, clips, seed0, prec="fp32", cfg=TRAIN):
    """Relative residual ||y1 - Phi_Y,S beta|| / ||y1|| of the learned
    selection (no fallback) on `clips` seeded clips."""
    import torch
    dev = torch.device("cuda", device)
    n, K = cfg["n"], cfg["K"]
    k = min(1000, 4 * n)
    b = np.array(blob, dtype=np.float32)
    b[8] = np.inf
    ctx = C.Context(device)
    C.cdmd_selector_load(ctx, torch.from_numpy(b).to(dev))
    out = []
    for c in range(clips):
        spec, r, cseed = clip_setup(seed0 + c, **cfg)
        D = C.cdmd_synth_clip(ctx, spec, seed0 + c)
        DY = C.cdmd_sketch(ctx, D, k, cseed, prec=prec)
        try:
            dec = C.cdmd_decompose(ctx, DY, r, K, selector="mlp", with_phiy=True)
            C.cdmd_status_sync(ctx)
        except C.CdmdError:
            continue
        out.append(_residual_fn(dec, DY)())
    return np.asarray(out)


def calibrate_tol(residuals, quantile=0.99, slack=1.25):
    """Fallback threshold: slack x the given quantile of the learned
    selection's relative residuals on the calibration clips, so that the
    sparse-coding solver takes over on the outliers."""
    r = np.asarray([x for x in residuals if np.isfinite(x)])
    return float(slack * np.quantile(r, quantile))


def save_model(path, blob, meta):
    with open(path, "w") as f:
        json.dump(dict(blob=[float(x) for x in blob], **meta), f, indent=1)


def load_model(path=DEFAULT_MODEL):
    """(blob float32 array, metadata dict) of a saved model."""
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d.pop("blob"), dtype=np.float32), d


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--clips", type=int, default=20000)
    t.add_argument("--calib-clips", type=int, default=500)
    t.add_argument("--seed0", type=int, default=1_000_000)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--batch", type=int, default=4096)
    t.add_argument("--lr", type=float, default=3e-3)
    t.add_argument("--lanes", type=int, default=8)
    t.add_argument("--device", type=int, default=0)
    t.add_argument("--out", default=DEFAULT_MODEL)
    t.add_argument("--labels", choices=["clean", "y1"], default="clean")
    a = ap.parse_args(argv)
    t0 = time.time()
    X, Y, meta = collect(a.device, a.clips, a.seed0, lanes=a.lanes, log_every=2000, labels=a.labels)
    skipped = list(getattr(collect, "skipped", []))
    t_collect = time.time() - t0
    print(f"collected {X.shape[0]} mode rows from {a.clips} clips in {t_collect:.1f} s", flush=True)
    t1 = time.time()
    blob, hist = train(X, Y, a.device, epochs=a.epochs, batch=a.batch, lr=a.lr, log=print)
    t_train = time.time() - t1
    cal_seed0 = a.seed0 + a.clips + 100_000
    Xc, Yc, _ = collect(a.device, a.calib_clips, cal_seed0, lanes=a.lanes, labels=a.labels)
    tol = calibrate_tol(learned_residuals(a.device, blob, a.calib_clips, cal_seed0))
    blob[8] = tol
    acc_train = accuracy(blob, X, Y, a.device)
    acc_cal = accuracy(blob, Xc, Yc, a.device)
    info = dict(train_clips=a.clips, seed0=a.seed0, skipped_clips=len(skipped), calib_clips=a.calib_clips, calib_seed0=cal_seed0,
                rows=int(X.shape[0]), epochs=a.epochs, batch=a.batch, lr=a.lr, loss_history=hist,
                accuracy_train=acc_train, accuracy_calib=acc_cal, tol=tol,
                labels=a.labels, tol_rule="1.25 x 99th percentile of the learned selection's relative residual "
                                          "on the calibration clips",
                train_config=TRAIN, collect_s=t_collect, train_s=t_train)
    save_model(a.out, blob, info)
    print(json.dumps({k: v for k, v in info.items() if k != "loss_history"}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
