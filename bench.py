#!/usr/bin/env python
"""Throughput benchmark: compressed-DMD background subtraction, frames/s.

Workload: seeded synthetic 1920x1080 grayscale clips of 200 frames
(textured low-rank background, 3 moving rectangles, +-10 % illumination
drift, noise sigma 3; k = 1000 Gaussian measurements drawn in-kernel from
Philox, target rank r = 20, K = 10 background modes, threshold 25 grey), five
per GPU (the others rendered on the device), all seen through one
measurement matrix C (one camera, one sensing matrix, video processed window
by window).  A step is one pass of the whole hot path over the five clips:
    sketch of all (frames widened to BF16 and packed 512 to a launch, one
    draw of C feeding every frame of it) -> per clip: decompose -> lift
    (selected modes) -> subtract + bit-pack.
value = frames processed by all ranks / wall time of the timed steps (max over
ranks); the clips (415 MB each) are resident in HBM and larger than L2, so
no flush is needed between steps.  Each pass is timed with CUDA events on the
launching stream; the sketch is the dominant kernel and carries the roofline.
--clips-per-step 1 times the one-clip step (no sharing of C).

e2e: the same metric through cdmd_run_host_shared with pinned host buffers
(every clip copied in and every mask copied out, every step).
cpu_baseline / --impl reference: the FP64 oracle on the host cores, on a
bounded pixel sample of the clip, scaled to the full frame.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x2|fp32]
       [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(width=1920, height=1080, n=200, k=1000, r=20, K=10, tau=25.0, drift=0.1, clip_seed=2024,
                c_seed=0x5EED1080, clips_per_step=5)
METRIC = "cDMD 1080p frames/s"
UNIT = "frames/s"


def workload_name(prec, selector="omp"):
    w = WORKLOAD
    return f"cdmd_{w['width']}x{w['height']}_n{w['n']}_k{w['k']}_r{w['r']}_K{w['K']}_gaussian_{prec}_{selector}"


def clip_seed(rank):
    """Each rank sketches its own clip (clips are independent): weak scaling,
    no collective on the data path."""
    return WORKLOAD["clip_seed"] + rank


def max_over_ranks(x, dist, device):
    """The slowest rank's time (the job's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank, world, seconds):
    """Frames of all ranks over the max-over-ranks time."""
    return world * frames_per_rank / seconds


def fmeasure(pred, truth):
    """F-measure of a boolean mask against the generator's ground truth."""
    tp = float(np.count_nonzero(pred & truth))
    fp = float(np.count_nonzero(pred & ~truth))
    fn = float(np.count_nonzero(~pred & truth))
    prec = tp / (tp + fp) if tp + fp > 0 else 0.0
    rec = tp / (tp + fn) if tp + fn > 0 else 0.0
    return 2 * prec * rec / (prec + rec) if prec + rec > 0 else 0.0


GOLDEN = os.path.join(ROOT, "tests", "golden", "cdmd_1080p_x200.json")


def load_golden():
    """The FP64 oracle's stored results for the 1920x1080x200 clip (written by
    tests/golden/make_fullsize_1080p.py), or None if absent."""
    if not os.path.exists(GOLDEN):
        return None
    with open(GOLDEN) as f:
        return json.load(f)


def golden_applies(gold, clip_seed_value):
    if gold is None:
        return False
    g, w = gold["workload"], WORKLOAD
    return (g["width"], g["height"], g["n"], g["clip_seed"], g["drift"], g["k"], g["c_seed"], g["r"], g["K"],
            g["tau"]) == (w["width"], w["height"], w["n"], clip_seed_value, w["drift"], w["k"], w["c_seed"],
                          w["r"], w["K"], w["tau"])


def compare_with_golden(gold, form, lam, sel, bg_at, F):
    """Errors of one run of the clip against the oracle's stored results:
    eigenvalues matched one to one (relative error, all modes and modes at
    least 1e-3 from any other), the selected set, the background at the
    stored seeded (pixel, frame) points (relative 2-norm and max abs error;
    bg_at(J, T) returns the run's background there) and the F-measure
    against truth beside the oracle's."""
    g = gold[form]
    lam_ref = np.array([complex(a, b) for a, b in gold["lam"]])
    idx = [int(np.argmin(np.abs(lam - x))) for x in lam_ref]
    rel = np.abs(lam[idx] - lam_ref) / np.abs(lam_ref)
    sep = np.array([np.min(np.abs(np.delete(lam_ref, i) - x)) >= 1e-3 for i, x in enumerate(lam_ref)])
    rng = np.random.default_rng(gold["bg_sample_seed"])
    m = gold["workload"]["width"] * gold["workload"]["height"]
    J = rng.integers(0, m, gold["bg_sample_count"])
    T = rng.integers(0, gold["workload"]["n"], gold["bg_sample_count"])
    ref = np.array(g["bg_samples"])
    got = bg_at(J, T)
    return {"oracle_form": form,
            "eig_rel_err_max_separated": float(rel[sep].max()) if sep.any() else None,
            "eig_rel_err_max_all": float(rel.max()), "eig_separated_modes": int(sep.sum()),
            "selection_equal": bool(len(set(idx)) == len(idx) and set(int(v) for v in sel) ==
                                    {idx[q] for q in g["sel"]}),
            "bg_rel_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "bg_max_abs_err_grey": float(np.abs(got - ref).max()),
            "bg_points": int(len(ref)),
            "fmeasure": F, "fmeasure_oracle": g["F"], "fmeasure_diff": abs(F - g["F"])}


def launches_per_step(selector, K, clips=1, n=200):
    """Kernels one pipeline step over `clips` clips of n frames launches:
    sketch 2 for one clip (tiles + fixed-order reduce), or for several clips
    under one C a widen pass per clip and 2 per packed launch of up to 512
    frames; per clip: decompose 15 (Gram 2, tridiagonalisation 1, eigenpairs 1,
    orthonormalise 1, back-transform 1, B 1, A~ 1, eig FP32 1, Newton 1,
    FP64 QR fallback 1, order 1, G 1, Gram-form H 1, selection 1) + 2 for the
    learned selection (scoring, least squares on its picks, then the OMP
    launch that exits at once unless the picks were rejected); lift one per
    16 modes; subtract 2 (lambda^t table + pass)."""
    sketch = 2 if clips == 1 else clips + 2 * (-(-clips * n // 512))
    return sketch + clips * (15 + (2 if selector == "mlp" else 0) + (K + 15) // 16 + 2)


def algorithmic_counts():
    """Per-step algorithmic work of each pass (minimum the method must do)."""
    w = WORKLOAD
    m, n, k, K = w["width"] * w["height"], w["n"], w["k"], w["K"]
    return dict(
        sketch_flops=2.0 * k * m * n,                       # C D, C never stored
        sketch_bytes=float(m * n),                          # D read once
        gaussians=float(k * m),
        lift_bytes=float(m * (n - 1) + m * K * 8),          # X' read, Phi (K complex64) written
        subtract_bytes=float(m * n + m * K * 8 + n * ((m + 31) // 32) * 4),
    )


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def source_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def dram_traffic(kernel_file):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, only
    if the kernel source has not changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    entry = table.get(kernel_file)
    src = os.path.join(ROOT, "paper_1512_04205_gb300", "csrc", kernel_file)
    if not entry or not os.path.exists(src) or entry.get("source_sha") != source_hash(src):
        return None
    return entry.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        # nvidia-smi's start-up takes driver locks that can stall CUDA calls:
        # wait for its first sample before the timed region begins
        import select
        self.first = ""
        ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
        if ready:
            self.first = self.proc.stdout.readline()
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "first", "") + out).strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ----------------------------------------------------------------------------

CPU_SAMPLE_PX = WORKLOAD["width"] * 8     # pixels per oracle step (eight rows of the frame)


def oracle_step(clip, sample_px):
    """One step of the FP64 oracle on a bounded sample of the clip, timed
    part by part: the sketch C D of the first `sample_px` pixels (k x n, the
    same shape as the full clip's sketch), the small solves on that sketch
    (the full-size problem: their cost does not depend on the pixel count),
    then lift, background and mask of those pixels.  Returns the measured
    seconds of each part and the full-clip estimate (pixel passes scaled by
    m / sample_px, small solves once)."""
    from oracle import cdmd as O
    from oracle import measurement as M
    w = WORKLOAD
    m, n, k, r, K = clip.m, clip.n, w["k"], w["r"], w["K"]
    Dm = clip.frames[:, :sample_px].T.astype(np.float64)
    t0 = time.perf_counter()
    Cs = M.gaussian_block(w["c_seed"], np.arange(k), np.arange(sample_px))
    DY = O.sketch(Cs, Dm)
    t1 = time.perf_counter()
    dec = O.decompose(DY, r, K)
    t2 = time.perf_counter()
    Phi = O.lift(Dm, dec["G"][:, dec["sel"]])
    bg = O.background(Phi, dec["beta"], dec["lam"][dec["sel"]], n)
    O.pack_mask(O.foreground_mask(Dm, bg, w["tau"]))
    t3 = time.perf_counter()
    scale = m / sample_px
    parts = dict(sketch_s=t1 - t0, decompose_s=t2 - t1, pixel_passes_s=t3 - t2)
    est = (parts["sketch_s"] + parts["pixel_passes_s"]) * scale + parts["decompose_s"]
    return dict(measured_s=t3 - t0, parts=parts, scale=scale, full_clip_estimate_s=est)


def oracle_sample_text(clip, sample_px, scale):
    return (f"per step: first {sample_px} of {clip.m} pixels x {clip.n} frames (sketch, lift, background, mask), "
            f"plus the small solves on that {WORKLOAD['k']}x{clip.n} sketch; full-clip figure = pixel passes x "
            f"{scale:.0f} + small solves (an estimate from the measured parts)")


def cpu_cores():
    return os.cpu_count() or 1


def run_reference(args, rank):
    """The oracle is the reference arm.  Each step runs oracle_step for real;
    ms_per_step is its measured time, `value` the full-clip frames/s estimate
    from the measured parts (labelled as such)."""
    if rank != 0:
        return 0
    import videogen
    w = WORKLOAD
    clip = videogen.make_clip(w["width"], w["height"], w["n"], seed=w["clip_seed"], drift=w["drift"])
    steps = []
    for i in range(args.warmup + args.steps):
        st = oracle_step(clip, CPU_SAMPLE_PX)
        if i >= args.warmup:
            steps.append(st)
    measured_ms = 1e3 * float(np.mean([st["measured_s"] for st in steps]))
    est_s = float(np.mean([st["full_clip_estimate_s"] for st in steps]))
    value = w["n"] / est_s
    sample = oracle_sample_text(clip, CPU_SAMPLE_PX, steps[0]["scale"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": measured_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.prec, args.selector), "m": clip.m, "n": w["n"], "k": w["k"],
                       "r": w["r"], "K": w["K"], "implementation": "FP64 CPU oracle, OMP selection"},
            "measured": {"ms_per_step": measured_ms, "what": "one oracle step on the sample (see cpu_baseline.sample)",
                         "parts_ms": {k2: 1e3 * float(np.mean([st["parts"][k2] for st in steps]))
                                      for k2 in steps[0]["parts"]}},
            "estimate": {"ms_per_clip_full": est_s * 1e3, "value_is_estimate": True,
                         "formula": "(sketch + pixel passes) x m / sample pixels + small solves"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# batch of clips of uneven size (grouped launches, captured graph, autotuned)
# ----------------------------------------------------------------------------

BATCH = dict(clips=64, sizes=[(320, 240), (640, 480), (1280, 720), (1920, 1080)], n_lo=50, n_hi=300, r_lo=10,
             r_hi=30, K=10, tau=25.0, seed=4242)


def run_batch_measure(C, SEL, torch, dev, args, model):
    """64 seeded clips (resolution, length and rank drawn per clip, k =
    min(1000, 4n)) rendered on the device, planned as one batch (grouped
    launches, graph, autotuner) and timed over replays; the same clips one
    after another through cdmd_run for comparison."""
    import videogen
    rng = np.random.default_rng(BATCH["seed"])
    clips, frames_total = [], 0
    ctx = C.Context(dev.index or 0)
    for i in range(BATCH["clips"]):
        w, h = BATCH["sizes"][int(rng.integers(0, len(BATCH["sizes"])))]
        n = int(rng.integers(BATCH["n_lo"], BATCH["n_hi"] + 1))
        r = int(rng.integers(BATCH["r_lo"], BATCH["r_hi"] + 1))
        spec = videogen.clip_spec(w, h, n, BATCH["seed"] * 1000 + i, drift=float(rng.uniform(0, 0.1)))
        D = C.cdmd_synth_clip(ctx, spec, BATCH["seed"] * 1000 + i)
        clips.append(dict(D=D, k=min(1000, 4 * n), r=r, K=min(BATCH["K"], r), seed=77 + i))
        frames_total += n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = C.Batch(clips, BATCH["tau"], prec=args.prec, selector=args.selector, autotune=True, grouped=True,
                    graph=True, lanes=8, selector_blob=model)
    plan_s = time.perf_counter() - t0
    tune = batch.tuning()
    reps = max(3, min(args.steps, 10))
    batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    batch.status_sync()
    ms = e0.elapsed_time(e1) / reps
    # the same clips one after another through the single-clip call
    if model is not None:
        C.cdmd_selector_load(ctx, model)
    params = [C.make_params(c["k"], c["r"], c["K"], BATCH["tau"], seed=c["seed"], prec=args.prec,
                            selector=args.selector) for c in clips]
    for c, p in zip(clips, params):
        C.cdmd_run(ctx, c["D"], p)
    torch.cuda.synchronize()
    e0.record()
    for c, p in zip(clips, params):
        C.cdmd_run(ctx, c["D"], p)
    e1.record()
    torch.cuda.synchronize()
    C.cdmd_status_sync(ctx)
    seq_ms = e0.elapsed_time(e1)
    pix_frames = sum(int(c["D"].shape[0]) * int(c["D"].shape[1]) for c in clips)
    batch.close()
    # the same batch as per-clip launches on lanes (one graph, no grouped passes)
    lanes_b = C.Batch(clips, BATCH["tau"], prec=args.prec, selector=args.selector, autotune=True, grouped=False,
                      graph=True, lanes=8, selector_blob=model)
    lanes_b.run()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        lanes_b.run()
    e1.record()
    torch.cuda.synchronize()
    lanes_b.status_sync()
    lanes_ms = e0.elapsed_time(e1) / reps
    lanes_tune = lanes_b.tuning()
    lanes_b.close()
    return {"clips": len(clips), "frames": frames_total, "pixel_frames": pix_frames,
            "value": frames_total / (ms * 1e-3), "unit": "frames/s", "ms_per_batch": ms,
            "gpixel_frames_per_s": pix_frames / (ms * 1e-3) / 1e9,
            "sequential_cdmd_run": {"value": frames_total / (seq_ms * 1e-3), "ms_per_batch": seq_ms},
            "per_clip_lanes": {"value": frames_total / (lanes_ms * 1e-3), "ms_per_batch": lanes_ms,
                               "tuning": lanes_tune},
            "tuning": tune, "plan_s": plan_s,
            "config": {"sizes": BATCH["sizes"], "n": [BATCH["n_lo"], BATCH["n_hi"]], "k": "min(1000, 4n)",
                       "r": [BATCH["r_lo"], BATCH["r_hi"]], "K": BATCH["K"], "launch": "grouped sketch + subtract "
                       "per wave of clips, per-clip small solves and lifts on lanes, one CUDA graph"}}


# ----------------------------------------------------------------------------
# Measurement-matrix study (Section 4: fps and F-measure against the number of
# samples p for Gaussian, sparse and single-pixel C on a 720x480x200 video;
# bootstrap confidence intervals of F over random draws of C)
# ----------------------------------------------------------------------------

STUDY = dict(width=720, height=480, n=200, p=[25, 50, 100, 200, 400, 700, 1000], seeds=12, K=10, tau=25.0,
             clip_seed=31, boot=4000)


def bootstrap_ci(values, rng, boot):
    """Percentile bootstrap 95 % interval of the mean."""
    v = np.asarray(values, dtype=np.float64)
    means = v[rng.integers(0, len(v), size=(boot, len(v)))].mean(axis=1)
    return [float(np.percentile(means, 2.5)), float(np.percentile(means, 97.5))]


def run_study(args):
    """One JSON line: per measurement type and p, the time of sketch +
    decompose + lift (the foreground mask excluded, as in the paper's study),
    the F-measure of the mask against the generator's truth, and its
    bootstrap interval over independent draws of C.  The rank is automatic
    (optimal hard threshold, at most min(32, p, n-1)) and K = 10 modes are
    selected by OMP, as in the paper's evaluation settings."""
    import torch

    import videogen
    from paper_1512_04205_gb300 import build
    from paper_1512_04205_gb300 import cdmd as C

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    S = STUDY
    clip = videogen.make_clip(S["width"], S["height"], S["n"], seed=S["clip_seed"], drift=0.1)
    m, n = clip.m, clip.n
    truth = clip.truth.T
    D = torch.from_numpy(clip.frames).to(dev)
    ctx = C.Context(0)
    stream = torch.cuda.current_stream()
    density = float(np.log(m) / m)      # sparsity factor s = m / log(m) (Section 4, evaluation settings)
    rng = np.random.default_rng(7)
    rows = []
    for ctype in ("gaussian", "sparse", "rowsample", "srft"):
        for p in S["p"]:
            r_max = min(32, p, n - 1)
            times, fs, ranks, build_ms = [], [], [], []
            for sd in range(S["seeds"] + 1):       # the first draw warms up and is not kept
                seed = 1000 * sd + p
                meas = None
                if ctype != "gaussian":
                    t0 = time.perf_counter()
                    meas = C.Measure(ctx, ctype, m, p, seed, density=density if ctype == "sparse" else 0.0)
                    torch.cuda.synchronize()
                    bms = (time.perf_counter() - t0) * 1e3
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev[0].record(stream)
                if meas is None:
                    DY = C.cdmd_sketch(ctx, D, p, seed, prec=args.prec)
                else:
                    DY = C.cdmd_sketch_gather(ctx, D, meas)
                ev[1].record(stream)
                dec, r, _ = C.cdmd_decompose_auto(ctx, DY, r_max, min(S["K"], r_max), selector="omp")
                ev[2].record(stream)
                Kc = min(S["K"], r)
                Phi = C.cdmd_lift(ctx, D, dec["G"][:r], cols=dec["sel"], ncols=Kc, prec=args.prec)
                ev[3].record(stream)
                mask = C.cdmd_subtract(ctx, D, Phi, dec["beta"][:r], dec["lam"][:r], S["tau"], cols=dec["sel"])
                C.cdmd_status_sync(ctx)
                if sd == 0:
                    continue
                times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
                fs.append(fmeasure(C.unpack_mask(mask, m), truth))
                ranks.append(r)
                if meas is not None:
                    build_ms.append(bms)
            per = np.median(np.array(times), axis=0)
            ms = float(np.median(np.array(times).sum(axis=1)))
            rows.append({"ctype": ctype, "p": p, "ms": ms, "fps": n / (ms * 1e-3),
                         "sketch_ms": float(per[0]), "decompose_ms": float(per[1]), "lift_ms": float(per[2]),
                         "F_mean": float(np.mean(fs)), "F_ci95": bootstrap_ci(fs, rng, S["boot"]),
                         "F_min": float(np.min(fs)), "F_max": float(np.max(fs)),
                         "rank_median": float(np.median(ranks)),
                         "build_ms": float(np.median(build_ms)) if build_ms else None})
    line = {"study": ("measurement matrices (Gaussian, sparse, single pixel, SRFT) against the number of "
                      "samples p"),
            "workload": f"synthetic {S['width']}x{S['height']}x{S['n']}, seed {S['clip_seed']}",
            "timing": ("CUDA events around sketch + decompose + lift (mask excluded), median over "
                       f"{S['seeds']} draws of C after one warm-up draw; the Gaussian C is drawn in the sketch "
                       "kernel, sparse and single-pixel C and the SRFT's kept frequencies are built on the device "
                       "beforehand (build_ms, host timed, not in ms); the SRFT sketch is an FFT pass"),
            "sparse_density": density, "precision": args.prec, "selector": "omp", "rank": "automatic",
            "K": S["K"], "tau": S["tau"], "draws_of_C": S["seeds"], "bootstrap": S["boot"], "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU path
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch

    import videogen
    from paper_1512_04205_gb300 import build
    from paper_1512_04205_gb300 import cdmd as C
    from paper_1512_04205_gb300 import selector as SEL

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOAD
    clip = videogen.make_clip(w["width"], w["height"], w["n"], seed=clip_seed(rank), drift=w["drift"])
    m, n, k, r, K = clip.m, clip.n, w["k"], w["r"], w["K"]
    D = torch.from_numpy(clip.frames).to(dev)
    main_stream = torch.cuda.current_stream()
    model = torch.from_numpy(SEL.load_model()[0]).to(dev) if args.selector == "mlp" else None

    cps = args.clips_per_step

    class Lane:
        """One step in flight: its own context (workspace), stream and the
        outputs of each of its clips."""

        def __init__(self, stream):
            self.ctx = C.Context(local_rank)
            self.stream = stream
            self.DY = [torch.empty((n, k), dtype=torch.float64, device=dev) for _ in range(cps)]
            self.dec = [C.decompose_outputs(n, k, r, K, dev) for _ in range(cps)]
            self.Phi = [torch.empty((m, K, 2), dtype=torch.float32, device=dev) for _ in range(cps)]
            self.mask = [torch.empty((n, (m + 31) // 32), dtype=torch.int32, device=dev) for _ in range(cps)]
            if model is not None:
                C.cdmd_selector_load(self.ctx, model, stream=stream)

    lanes = [Lane(main_stream)] + [Lane(torch.cuda.Stream(device=dev)) for _ in range(max(0, args.inflight - 1))]
    ctx = lanes[0].ctx
    mask = lanes[0].mask[0]
    # the step's other clips: same size, own content, rendered on the device
    Ds = [D]
    for i in range(1, cps):
        sd = clip_seed(rank) + 1000 * i
        Ds.append(C.cdmd_synth_clip(ctx, videogen.clip_spec(w["width"], w["height"], n, sd, drift=w["drift"]), sd))
    torch.cuda.synchronize()

    def step(prec, selector, events=None, lane=None):
        L = lane or lanes[0]
        st = L.stream
        with torch.cuda.stream(st):
            if events is not None:
                events[0].record(st)
            if cps == 1:
                C.cdmd_sketch(L.ctx, D, k, w["c_seed"], prec=prec, DY=L.DY[0])
            else:
                C.cdmd_sketch_shared(L.ctx, Ds, k, w["c_seed"], prec=prec, DYs=L.DY)
            if events is not None:
                events[1].record(st)
            for i in range(cps):
                C.cdmd_decompose(L.ctx, L.DY[i], r, K, selector=selector, out=L.dec[i])
            if events is not None:
                events[2].record(st)
            for i in range(cps):
                C.cdmd_lift(L.ctx, Ds[i], L.dec[i]["G"], cols=L.dec[i]["sel"], ncols=K, prec=prec, Phi=L.Phi[i])
            if events is not None:
                events[3].record(st)
            for i in range(cps):
                C.cdmd_subtract(L.ctx, Ds[i], L.Phi[i], L.dec[i]["beta"], L.dec[i]["lam"], w["tau"],
                                cols=L.dec[i]["sel"], mask=L.mask[i])
            if events is not None:
                events[4].record(st)
    stream = main_stream

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, selector, steps, warmup, sample_clocks):
        for _ in range(warmup):
            step(prec, selector)
        C.cdmd_status_sync(ctx)
        barrier()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(gpu_index(local_rank)) if sample_clocks else None
        if sampler:
            sampler.start()
        start.record(stream)
        for s in range(steps):
            step(prec, selector, evs[s])
        end.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        C.cdmd_status_sync(ctx)
        total_ms = start.elapsed_time(end)
        passes = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs]).mean(axis=0) / cps
        total_ms = max_over_ranks(total_ms, dist, dev)
        barrier()
        return total_ms, passes, clocks

    def pipelined(prec, selector, steps, warmup, sample_clocks):
        """Whole-job throughput with len(lanes) clips in flight (one per stream)."""
        for L in lanes:
            C.cdmd_set_sm_limit(L.ctx, args.sm_limit)
        for i in range(warmup):
            step(prec, selector, lane=lanes[i % len(lanes)])
        for L in lanes:
            C.cdmd_status_sync(L.ctx, L.stream)
        barrier()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(gpu_index(local_rank)) if sample_clocks else None
        if sampler:
            sampler.start()
        start.record(main_stream)
        for L in lanes[1:]:
            L.stream.wait_event(start)
        for i in range(steps):
            step(prec, selector, lane=lanes[i % len(lanes)])
        for L in lanes[1:]:
            ev = torch.cuda.Event()
            ev.record(L.stream)
            main_stream.wait_event(ev)
        end.record(main_stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        for L in lanes:
            C.cdmd_status_sync(L.ctx, L.stream)
            C.cdmd_set_sm_limit(L.ctx, 0)
        total_ms = start.elapsed_time(end)
        total_ms = max_over_ranks(total_ms, dist, dev)
        barrier()
        return total_ms, clocks

    def median_postpass():
        """The mask post-pass (3 x 3 median filter of each frame) on the mask
        the last step left, timed alone after an L2 flush per launch."""
        out = torch.empty_like(mask)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        with torch.cuda.stream(main_stream):
            for _ in range(3):
                C.cdmd_median3x3(ctx, mask, w["width"], w["height"], out=out)
            for e0, e1 in evs:
                flush.zero_()
                e0.record(main_stream)
                C.cdmd_median3x3(ctx, mask, w["width"], w["height"], out=out)
                e1.record(main_stream)
        torch.cuda.synchronize()
        us = float(np.median([e0.elapsed_time(e1) for e0, e1 in evs])) * 1e3
        return us, C.unpack_mask(out, m)

    def exact_comparator(prec, steps, warmup):
        """Exact DMD on the same clip (snapshot Gram, decompose from the Gram,
        lift, subtract; OMP selection), one clip per step on one stream: the
        comparator the paper times cDMD against."""
        L = lanes[0]
        R = torch.empty((n, n), dtype=torch.float64, device=dev)
        dec = C.decompose_outputs(n, k, r, K, dev)
        emask = torch.empty_like(mask)

        def one(ev=None):
            with torch.cuda.stream(main_stream):
                if ev is not None:
                    ev[0].record(main_stream)
                C.cdmd_snapshot_gram(ctx, D, R=R)
                if ev is not None:
                    ev[1].record(main_stream)
                C.cdmd_decompose_gram(ctx, R, r, K, out=dec)
                if ev is not None:
                    ev[2].record(main_stream)
                C.cdmd_lift(ctx, D, dec["G"], cols=dec["sel"], ncols=K, prec=prec, Phi=L.Phi[0])
                if ev is not None:
                    ev[3].record(main_stream)
                C.cdmd_subtract(ctx, D, L.Phi[0], dec["beta"], dec["lam"], w["tau"], cols=dec["sel"], mask=emask)
                if ev is not None:
                    ev[4].record(main_stream)
        for _ in range(warmup):
            one()
        C.cdmd_status_sync(ctx)
        barrier()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        for e in evs:
            one(e)
        torch.cuda.synchronize()
        C.cdmd_status_sync(ctx)
        total_ms = sum(e[0].elapsed_time(e[4]) for e in evs)
        passes = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs]).mean(axis=0)
        return dict(total_ms=max_over_ranks(total_ms, dist, dev), passes=passes, mask=C.unpack_mask(emask, m))

    def auto_rank_measure():
        """The rank the optimal hard threshold picks on this clip's sketch
        (Remark 2) and the time of the decomposition that picks it (one call,
        including its host synchronisation), beside the fixed-rank one."""
        L = lanes[0]
        with torch.cuda.stream(main_stream):
            C.cdmd_sketch(ctx, D, k, w["c_seed"], prec=args.prec, DY=L.DY[0])
            times = []
            for i in range(4):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(main_stream)
                _, r_auto, tau = C.cdmd_decompose_auto(ctx, L.DY[0], min(32, k, n - 1), K, selector="omp")
                e1.record(main_stream)
                torch.cuda.synchronize()
                if i:
                    times.append(e0.elapsed_time(e1))
        C.cdmd_status_sync(ctx)
        return {"rank": r_auto, "tau": tau, "r_max": min(32, k, n - 1), "decompose_auto_ms": float(np.median(times)),
                "note": "rank chosen on the device from the sketch of the benchmark clip; the headline keeps r = "
                        f"{r} as its workload fixes"}

    def rademacher_measure():
        """The step's sketch with Rademacher C instead of Gaussian: +-1 is
        exact in BF16, so one tensor product instead of hi + lo, and one Philox
        counter gives a pixel's 128 rows.  Timed over the same clips, per clip,
        against the tensor peak (2 k m n flop per clip)."""
        L = lanes[0]
        evs = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        with torch.cuda.stream(main_stream):
            for _ in range(2):
                C.cdmd_sketch_shared(ctx, Ds, k, w["c_seed"], ctype="rademacher", prec=args.prec, DYs=L.DY)
            evs[0].record(main_stream)
            for _ in range(args.steps):
                C.cdmd_sketch_shared(ctx, Ds, k, w["c_seed"], ctype="rademacher", prec=args.prec, DYs=L.DY)
            evs[1].record(main_stream)
        torch.cuda.synchronize()
        C.cdmd_status_sync(ctx)
        ms = evs[0].elapsed_time(evs[1]) / (args.steps * cps)
        tf = 2.0 * k * m * n / (ms * 1e-3) / 1e12
        peak = float(load_peaks()[0].get("bf16_tflops_sustained", load_peaks()[0]["bf16_tflops"]))
        return {"sketch_ms_per_clip": ms, "tflops": tf, "frac": tf / peak, "peak_tflops": peak,
                "bytes_gbs": m * n / (ms * 1e-3) / 1e9,
                "form": (f"{cps} clips under one Rademacher C, packed 512 frames to a launch; the uint8 frames "
                         "converted to FP16 inside the kernel (no BF16 copies); time per clip includes the reduces; "
                         "one FP16 product (C exact)")}

    def gather_4k_measure(reps=5):
        """The gather workload: a 3840x2160 clip of 300 frames (8 moving
        ellipses) rendered on the device, sketched by sparse +-1 C (density
        1/1000) and by single-pixel C (k = 1000 pixels), then decompose
        (r = 30, K = 10), lift of the selected modes and subtract.  Each pass
        is timed with CUDA events on the launching stream (median of `reps`
        runs, each after an L2 flush) against its algorithmic bytes."""
        W4, H4, n4, k4, r4, K4 = 3840, 2160, 300, 1000, 30, 10
        m4 = W4 * H4
        spec = videogen.clip_spec(W4, H4, n4, 4321, n_objects=8, shape="ellipse")
        D4 = C.cdmd_synth_clip(ctx, spec, 4321)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        hbm = float(load_peaks()[0]["hbm_gbs"])
        out = {"workload": f"{W4}x{H4}x{n4}, 8 ellipses, k={k4}, r={r4}, K={K4}",
               "lift_precision": (f"{args.prec} (tensor cores: two frame chunks of at most 255, the second adding "
                                  "into Phi)" if args.prec == "bf16x2" else args.prec),
               "subtract": "tensor cores, two frame chunks of 150"}
        words = n4 * ((m4 + 31) // 32) * 4
        alg = {"lift": m4 * (n4 - 1) + m4 * K4 * 8, "subtract": m4 * n4 + m4 * K4 * 8 + words}
        for name, meas in (("sparse", C.Measure(ctx, "sparse", m4, k4, 77, 1e-3)),
                           ("single_pixel", C.Measure(ctx, "rowsample", m4, k4, 3))):
            alg_sk = m4 * n4 if name == "sparse" else k4 * n4
            times = {"sketch": [], "decompose": [], "lift": [], "subtract": []}
            for it in range(reps + 1):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
                with torch.cuda.stream(main_stream):
                    flush.zero_()
                    ev[0].record(main_stream)
                    DY4 = C.cdmd_sketch_gather(ctx, D4, meas)
                    ev[1].record(main_stream)
                    dec4 = C.cdmd_decompose(ctx, DY4, r4, K4)
                    ev[2].record(main_stream)
                    flush.zero_()
                    e_l = torch.cuda.Event(enable_timing=True)
                    e_l.record(main_stream)
                    Phi4 = C.cdmd_lift(ctx, D4, dec4["G"], cols=dec4["sel"], ncols=K4, prec=args.prec)
                    ev[3].record(main_stream)
                    flush.zero_()
                    e_s = torch.cuda.Event(enable_timing=True)
                    e_s.record(main_stream)
                    C.cdmd_subtract(ctx, D4, Phi4, dec4["beta"], dec4["lam"], w["tau"], cols=dec4["sel"])
                    ev[4].record(main_stream)
                torch.cuda.synchronize()
                if it == 0:
                    continue                      # warm-up (workspace growth)
                times["sketch"].append(ev[0].elapsed_time(ev[1]))
                times["decompose"].append(ev[1].elapsed_time(ev[2]))
                times["lift"].append(e_l.elapsed_time(ev[3]))
                times["subtract"].append(e_s.elapsed_time(ev[4]))
            C.cdmd_status_sync(ctx)
            med = {kk: float(np.median(v)) for kk, v in times.items()}
            rec = {"ms": med, "nnz": int(meas.nnz) if name == "sparse" else None}
            for pss, b in (("sketch", alg_sk), ("lift", alg["lift"]), ("subtract", alg["subtract"])):
                gbs = b / (med[pss] * 1e-3) / 1e9
                rec[pss + "_bytes"] = b
                rec[pss + "_gbs"] = gbs
                rec[pss + "_frac_hbm"] = gbs / hbm
            rec["frames_per_s_single_stream"] = n4 / (sum(med.values()) * 1e-3)
            out[name] = rec
        del D4, flush
        torch.cuda.empty_cache()
        return out

    def selector_eval(n_clips=10):
        """The learned selector on held-out clips of the workload's size
        (seeds outside its training and calibration ranges), against OMP on
        the same BF16 hi+lo sketch: fallbacks, identical selections, the
        background difference of the two forms (relative 2-norm on 20,000
        seeded pixels x all frames) and the F-measure of each against the
        generator's truth."""
        sctx = C.Context(local_rank)
        octx = C.Context(local_rank)
        if model is None:
            return None
        C.cdmd_selector_load(sctx, model)
        C.cdmd_selector_fallbacks(sctx, reset=True)
        J = torch.from_numpy(np.unique(np.random.default_rng(12).integers(0, m, 20_000))).to(dev)
        shifts = torch.arange(32, device=dev, dtype=torch.int32)

        def fm(mask_words, truth_dev):
            bits = ((mask_words.unsqueeze(-1) >> shifts) & 1).reshape(n, -1)[:, :m].bool()
            tp = int((bits & truth_dev).sum())
            fp = int((bits & ~truth_dev).sum())
            fn = int((~bits & truth_dev).sum())
            pr = tp / max(tp + fp, 1)
            rc = tp / max(tp + fn, 1)
            return 2 * pr * rc / (pr + rc) if pr + rc > 0 else 0.0

        def form(cx, Dc, dec):
            Phi = C.cdmd_lift(cx, Dc, dec["G"], cols=dec["sel"], ncols=K, prec=args.prec)
            mask_w = C.cdmd_subtract(cx, Dc, Phi, dec["beta"], dec["lam"], w["tau"], cols=dec["sel"])
            _, bgf = C.cdmd_subtract(cx, Dc, Phi, dec["beta"], dec["lam"], w["tau"], cols=dec["sel"], want_bg=True)
            out = (mask_w, bgf[:, J].double())
            del bgf
            return out

        rows = []
        for i in range(n_clips):
            sd = 7_000_000 + i
            spec = videogen.clip_spec(w["width"], w["height"], n, sd, drift=w["drift"])
            Dc = C.cdmd_synth_clip(octx, spec, sd)
            DYc = C.cdmd_sketch(octx, Dc, k, w["c_seed"], prec=args.prec)
            dm = C.cdmd_decompose(sctx, DYc, r, K, selector="mlp")
            do = C.cdmd_decompose(octx, DYc, r, K, selector="omp")
            mm, bm = form(sctx, Dc, dm)
            mo, bo = form(octx, Dc, do)
            C.cdmd_status_sync(sctx)
            C.cdmd_status_sync(octx)
            truth = torch.from_numpy(videogen.truth_from_spec(spec)).to(dev)
            rows.append({"seed": sd,
                         "same_set": sorted(dm["sel"].tolist()) == sorted(do["sel"].tolist()),
                         "bg_rel_diff_learned_vs_omp": float(torch.linalg.norm(bm - bo) / torch.linalg.norm(bo)),
                         "F_learned": fm(mm, truth), "F_omp": fm(mo, truth)})
            del Dc, truth
        fb = C.cdmd_selector_fallbacks(sctx)
        torch.cuda.empty_cache()
        return {"clips": n_clips, "size": f"{w['width']}x{w['height']}x{n}, k={k}, r={r}, K={K}",
                "seeds": "7000000 + i (outside training 1000000.. and calibration 1120000..)",
                "fallbacks": fb, "fallback_rate": fb / n_clips,
                "identical_selections": sum(q["same_set"] for q in rows),
                "F_learned_mean": float(np.mean([q["F_learned"] for q in rows])),
                "F_omp_mean": float(np.mean([q["F_omp"] for q in rows])),
                "bg_rel_diff_max": float(max(q["bg_rel_diff_learned_vs_omp"] for q in rows)),
                "per_clip": rows,
                "note": ("background error against the FP64 oracle's OMP result: tests/test_gpu_selector_1080p.py; "
                         "both forms use the same sketch")}

    # the headline form and the plain FP32 + OMP form it is compared with
    forms = {"head": (args.prec, args.selector)}
    if not args.no_plain and (args.prec, args.selector) != ("fp32", "omp"):
        forms["plain"] = ("fp32", "omp")
    results = {}
    gold = load_golden()
    check_gold = rank == 0 and golden_applies(gold, clip_seed(rank))

    def vs_oracle(selector, mk):
        """Clip 0 of lanes[0] (the stored oracle clip) against the oracle."""
        L = lanes[0]
        dec = L.dec[0]
        _, bg = C.cdmd_subtract(ctx, D, L.Phi[0], dec["beta"], dec["lam"], w["tau"], cols=dec["sel"],
                                want_bg=True)
        torch.cuda.synchronize()

        def bg_at(J, T):
            return bg[torch.from_numpy(T).to(dev), torch.from_numpy(J).to(dev)].double().cpu().numpy()
        out = compare_with_golden(gold, "mlp" if selector == "mlp" else "omp",
                                  torch.view_as_complex(dec["lam"]).cpu().numpy(), dec["sel"].cpu().numpy(), bg_at,
                                  fmeasure(mk, clip.truth.T))
        del bg
        return out

    for label, (prec, selector) in forms.items():
        total_ms, passes, clocks = timed(prec, selector, args.steps, args.warmup, sample_clocks=(label == "head"))
        results[label] = dict(total_ms=total_ms, passes=passes, clocks=clocks, mask=C.unpack_mask(mask, m))
        if check_gold:
            results[label]["vs_oracle"] = vs_oracle(selector, results[label]["mask"])
    fallbacks = None
    if args.selector == "mlp":
        fallbacks = sum(C.cdmd_selector_fallbacks(L.ctx, reset=True, stream=L.stream) for L in lanes)

    piped_ms, piped_clocks = (pipelined(args.prec, args.selector, args.steps, args.warmup, True) if len(lanes) > 1
                              else (None, None))

    # end to end through the public host-buffer call
    e2e = None
    if not args.no_e2e:
        # the public host-buffer call, one host thread per in-flight clip (each
        # with its own context and stream), so one clip's copies overlap the
        # others' compute; every step copies the clip in and the mask out
        import threading
        params = C.make_params(k, r, K, w["tau"], seed=w["c_seed"], prec=args.prec, selector=args.selector)
        hosts = [torch.from_numpy(clip.frames).pin_memory()] + [Dx.cpu().pin_memory() for Dx in Ds[1:]]
        hmasks = [[torch.empty((n, (m + 31) // 32), dtype=torch.int32).pin_memory() for _ in range(cps)]
                  for _ in lanes]
        for L in lanes:
            C.cdmd_set_sm_limit(L.ctx, args.sm_limit if len(lanes) > 1 else 0)
        errors = []

        def worker(i, count):
            try:
                for _ in range(count):
                    if cps == 1:
                        C.cdmd_run_host(lanes[i].ctx, hosts[0], params, mask_host=hmasks[i][0],
                                        stream=lanes[i].stream)
                    else:
                        C.cdmd_run_host_shared(lanes[i].ctx, hosts, params, mask_hosts=hmasks[i],
                                               stream=lanes[i].stream)
            except Exception as e:          # reported after the join
                errors.append(e)

        def run_all(count):
            ths = [threading.Thread(target=worker, args=(i, count)) for i in range(len(lanes))]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
            if errors:
                raise errors[0]

        run_all(1)
        barrier()
        # at least 4 calls per host thread, so the first and last calls (one
        # thread's lone copies and solves) weigh little in the total
        per_lane = max(4, -(-max(args.steps, len(lanes)) // len(lanes)))
        e2e_steps = per_lane * len(lanes)
        t0 = time.perf_counter()
        run_all(per_lane)
        dt = time.perf_counter() - t0
        for L in lanes:
            C.cdmd_set_sm_limit(L.ctx, 0)
        dt = max_over_ranks(dt, dist, dev)
        e2e = {"value": world * cps * n * e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": int(cps * m * n),
               "d2h_bytes_per_step": int(cps * n * ((m + 31) // 32) * 4), "steps": e2e_steps,
               "clips_per_step": cps, "host_threads": len(lanes),
               "api": ("cdmd_run_host" if cps == 1 else "cdmd_run_host_shared") +
                      " (pinned host videos in, host masks out)"}

    # measured after the headline, pipelined and end-to-end runs, so they see
    # the same device state as before these extra passes existed: the mask
    # post-pass on the head form's mask (the last pipelined step left it in
    # lanes[0]) and the exact-DMD comparator
    if piped_ms is None:
        step(args.prec, args.selector)   # the head form's mask, whatever form ran last
    results["median"] = median_postpass()
    exact = exact_comparator(args.prec, args.steps, args.warmup) if not args.no_exact else None
    rank_line = auto_rank_measure()
    rad_line = rademacher_measure() if args.prec == "bf16x2" else None

    batch_line = run_batch_measure(C, SEL, torch, dev, args, model) if not args.no_batch else None
    gather_line = gather_4k_measure() if not args.no_gather else None
    sel_line = selector_eval() if (args.selector == "mlp" and not args.no_selector_eval) else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    head = results["head"]
    steps = args.steps
    latency_value = job_throughput(cps * n * steps, world, head["total_ms"] * 1e-3)
    value = job_throughput(cps * n * steps, world, piped_ms * 1e-3) if piped_ms is not None else latency_value
    counts = algorithmic_counts()
    peaks, peak_src = load_peaks()
    sketch_ms = float(head["passes"][0])
    if args.prec == "bf16x2":
        # the method's work, 2 k m n per clip (C D); the hi + lo split doubles
        # the tensor products the kernel issues, reported apart as pipe work
        achieved = counts["sketch_flops"] / (sketch_ms * 1e-3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
        hbm_gbs = float(peaks["hbm_gbs"])
        t_ideal = max(counts["sketch_flops"] / (peak * 1e12), counts["sketch_bytes"] / (hbm_gbs * 1e9))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": t_ideal / (sketch_ms * 1e-3),
                "ideal_ms": t_ideal * 1e3, "measured_ms": sketch_ms,
                "flops_per_launch_unit": "2 k m n per clip (method's flops; hi + lo products not counted)",
                "tensor_pipe_tflops_hi_lo": 2.0 * achieved,
                "tensor_pipe_frac_hi_lo": 2.0 * achieved / peak,
                "traffic": dram_traffic("sketch_tc.cu"),
                "kernel": ("sketch (tcgen05 BF16 hi+lo" + (f", {cps} clips under one C packed 512 frames to a "
                                                           "launch; time per clip includes the widen passes and "
                                                           "the reduces)" if cps > 1
                                                           else "; time includes the reduce)")),
                "peak_source": (f"{peak_src} bf16 sustained (cuBLAS BF16 GEMM under the power cap, "
                                "MEASURED_PEAKS.json); frac = max(flop time at that peak, byte time at measured "
                                "HBM) / measured time")}
    else:
        fp32_peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        achieved = counts["sketch_flops"] / (sketch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": dram_traffic("sketch_fp32.cu"),
                "kernel": "sketch (FP32 FMA)", "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    per_pass = {name: float(v) for name, v in zip(["sketch", "decompose", "lift", "subtract"], head["passes"])}
    hbm = float(peaks["hbm_gbs"])
    lift_gbs = counts["lift_bytes"] / (per_pass["lift"] * 1e-3) / 1e9
    sub_gbs = counts["subtract_bytes"] / (per_pass["subtract"] * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup,
            "ms_per_step": (piped_ms if piped_ms is not None else head["total_ms"]) / steps,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.prec == "bf16x2" else "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.prec, args.selector), "selector": args.selector, "m": m, "n": n, "k": k, "r": r, "K": K,
                       "tau": w["tau"], "clips_per_step": cps,
                       "measurement": ("gaussian (Philox4x32-10, in-kernel); one C for all clips"
                                       + (", one draw of C feeds every frame of a packed launch"
                                          if cps > 1 else "")),
                       "precision": ("sketch BF16 hi+lo, lift FP16 hi+lo (G scaled per mode) on tcgen05, FP32 "
                                     "accumulation; FP64 small solves"
                                     if args.prec == "bf16x2" else "sketch+lift FP32 FMA; FP64 small solves"),
                       "l2": f"clip {m * n / 1e6:.0f} MB each vs 129 MB L2 (no flush)",
                       "parallelism": (f"clips x{world * cps} ({cps} per GPU per step), {len(lanes)} steps in flight "
                                       "per GPU (one stream each)"),
                       "sm_limit": args.sm_limit},
            "single_stream": {"value": latency_value, "ms_per_clip": head["total_ms"] / (steps * cps)},
            "per_pass_ms": per_pass,
            "pass_roofline": {"lift_gbs": lift_gbs, "lift_frac_hbm": lift_gbs / hbm, "subtract_gbs": sub_gbs,
                              "subtract_frac_hbm": sub_gbs / hbm, "hbm_peak_gbs": hbm},
            "roofline": roof,
            "gpu_launches": launches_per_step(args.selector, K, cps, n) * steps,
            "e2e": e2e}
    if piped_clocks is not None:
        line["clocks"] = piped_clocks
    elif head["clocks"] is not None:
        line["clocks"] = head["clocks"]
    truth = clip.truth.T
    line["accuracy"] = {"fmeasure_vs_truth": fmeasure(head["mask"], truth),
                        "selector": args.selector, "selector_fallbacks": fallbacks,
                        "selector_model": os.path.relpath(SEL.DEFAULT_MODEL, ROOT) if args.selector == "mlp" else None}
    if "vs_oracle" in head:
        line["accuracy"]["vs_oracle"] = head["vs_oracle"]
        line["accuracy"]["vs_oracle_note"] = ("clip 0 of the step against the FP64 oracle's stored results for the "
                                              "same uint8 clip (" + os.path.relpath(GOLDEN, ROOT) + ")")
    if "plain" in results:
        plain = results["plain"]
        agree = plain["mask"] == head["mask"]
        line["accuracy"]["plain_fp32_omp_fmeasure_vs_truth"] = fmeasure(plain["mask"], truth)
        line["plain_fp32"] = {"value": world * cps * n * steps / (plain["total_ms"] * 1e-3),
                              "ms_per_step": plain["total_ms"] / steps,
                              "per_pass_ms": {nm: float(v) for nm, v in
                                              zip(["sketch", "decompose", "lift", "subtract"], plain["passes"])},
                              "mask_agreement_vs_head": float(agree.mean())}
        if "vs_oracle" in plain:
            line["accuracy"]["plain_fp32_omp_vs_oracle"] = plain["vs_oracle"]
    med_us, med_mask = results["median"]
    med_bytes = 2 * n * ((m + 31) // 32) * 4
    line["postpass"] = {"kernel": "median3x3 (bit-sliced 3x3 median of each mask frame, zero padding)",
                        "us_per_clip": med_us, "gbs": med_bytes / (med_us * 1e-6) / 1e9,
                        "frac_hbm": med_bytes / (med_us * 1e-6) / 1e9 / hbm, "bytes": med_bytes,
                        "fmeasure_vs_truth_after": fmeasure(med_mask, truth),
                        "timing": "median of 10 launches, each after a 256 MB L2 flush; not in the step"}
    if exact is not None:
        t_gram = float(exact["passes"][0]) * 1e-3
        gram_tf = 2.0 * m * n * n / t_gram / 1e12
        bf16_peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
        exact_value = n * steps / (exact["total_ms"] * 1e-3)
        line["exact_dmd"] = {
            "value": exact_value, "unit": UNIT, "ms_per_clip": exact["total_ms"] / steps,
            "per_pass_ms": {nm: float(v) for nm, v in zip(["snapshot_gram", "decompose", "lift", "subtract"],
                                                           exact["passes"])},
            "gram_roofline": {"tflops": gram_tf, "frac_f16": gram_tf / bf16_peak,
                              "peak_note": "FP16 operands; dense FP16 and BF16 share the measured BF16 peak",
                              "gbs": m * n / t_gram / 1e9, "frac_hbm": m * n / t_gram / 1e9 / hbm,
                              "flops": 2.0 * m * n * n, "bytes": m * n},
            "cdmd_single_stream_over_exact": latency_value / exact_value,
            "fmeasure_vs_truth": fmeasure(exact["mask"], truth),
            "form": ("snapshot Gram D^T D on tcgen05 (uint8 exact in FP16, FP32 accumulation, FP64 reduce); "
                     f"FP64 small solves from the Gram; OMP; {args.prec} lift; one clip per step, one stream")}
    line["auto_rank"] = rank_line
    if rad_line is not None:
        line["rademacher_sketch"] = rad_line
    if batch_line is not None:
        line["batch"] = batch_line
    if gather_line is not None:
        line["gather_4k"] = gather_line
    if sel_line is not None:
        line["selector_eval"] = sel_line
    if not args.no_cpu:
        st = oracle_step(clip, CPU_SAMPLE_PX)
        line["cpu_baseline"] = {"value": w["n"] / st["full_clip_estimate_s"], "unit": UNIT, "cores": cpu_cores(),
                                "kind": "oracle", "sample": oracle_sample_text(clip, CPU_SAMPLE_PX, st["scale"]),
                                "measured_s": st["measured_s"],
                                "parts_s": st["parts"], "value_is_estimate": True,
                                "threads": "numpy elementwise single-threaded, BLAS multi-threaded"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["bf16x2", "fp32"], default="bf16x2")
    ap.add_argument("--selector", choices=["mlp", "omp", "lstsq"], default="mlp",
                    help="mode selection: learned (OMP fallback), OMP, or least squares on all modes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--inflight", type=int, default=12, help="steps in flight per GPU (streams)")
    ap.add_argument("--clips-per-step", type=int, choices=range(1, 9), default=WORKLOAD["clips_per_step"],
                    help="clips per step, all under one C (>= 2: their frames are packed 512 to a sketch "
                         "launch, so one draw of C feeds all of them)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batch of 64 clips of mixed size (grouped launches, graph, autotuner)")
    ap.add_argument("--no-selector-eval", action="store_true",
                    help="skip the learned selector's evaluation on held-out clips of the workload's size")
    ap.add_argument("--no-gather", action="store_true",
                    help="skip the 3840x2160x300 gather workload (sparse and single-pixel C)")
    ap.add_argument("--size", default=None,
                    help="WxH of a smaller clip for profiling captures (default: the 1920x1080 workload)")
    ap.add_argument("--sm-limit", type=int, default=136,
                    help="SMs the full-data passes of each in-flight clip may fill (0 = all)")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-DMD comparator")
    ap.add_argument("--study", action="store_true",
                    help="run the measurement-matrix study (p sweep of Gaussian, sparse and single-pixel C on "
                         "720x480x200, F-measure with bootstrap intervals) instead of the benchmark")
    args = ap.parse_args()
    if args.size:
        wd, ht = (int(v) for v in args.size.lower().split("x"))
        WORKLOAD.update(width=wd, height=ht)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.study:
        return run_study(args)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
