"""Host-side logic of bench.py (no GPU): launch counting, throughput
arithmetic, the F-measure, the bootstrap interval of the study, and the rule
that a DRAM-traffic figure is reported only for the kernel source it was
captured from."""
import json
import os

import numpy as np
import pytest

import bench


def test_launches_per_step_counts():
    # five clips of 200 frames under one C: 5 widen passes + 2 packed launches
    # with their reduces (1000 frames = 512 + 488), then per clip decompose
    # 15 + 2 (learned selector), lift 1, subtract 2
    assert bench.launches_per_step("mlp", 10, clips=5, n=200) == 9 + 5 * 20
    # one clip: sketch + reduce, decompose 15, lift 1, subtract 2
    assert bench.launches_per_step("omp", 10, clips=1, n=200) == 2 + 15 + 1 + 2
    # 17..32 modes take a second lift launch
    assert bench.launches_per_step("omp", 20, clips=1, n=200) == 2 + 15 + 2 + 2


def test_job_throughput_is_whole_job():
    # 2 ranks x 1000 frames in 0.5 s (the slowest rank's time)
    assert bench.job_throughput(1000, 2, 0.5) == 4000.0


def test_fmeasure_hand_counts():
    truth = np.array([1, 1, 1, 0, 0, 0, 0, 0], dtype=bool)
    pred = np.array([1, 1, 0, 1, 0, 0, 0, 0], dtype=bool)
    # tp 2, fp 1, fn 1: precision = recall = 2/3
    assert abs(bench.fmeasure(pred, truth) - 2 / 3) < 1e-12
    assert bench.fmeasure(np.zeros(8, dtype=bool), truth) == 0.0


def test_bootstrap_interval():
    rng = np.random.default_rng(0)
    assert bench.bootstrap_ci([0.5] * 12, rng, 500) == [0.5, 0.5]
    v = rng.normal(0.6, 0.05, size=12)
    lo, hi = bench.bootstrap_ci(v, rng, 4000)
    assert v.min() <= lo < v.mean() < hi <= v.max()
    # about 1.96 standard errors each side
    se = v.std(ddof=1) / np.sqrt(len(v))
    assert 2.5 * se < hi - lo < 5.0 * se


def test_study_settings():
    S = bench.STUDY
    assert (S["width"], S["height"], S["n"]) == (720, 480, 200)
    assert all(1 <= p <= 1000 for p in S["p"]) and S["p"] == sorted(S["p"])
    assert S["seeds"] >= 10 and S["K"] == 10


def test_traffic_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1512_04205_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k.cu"
    src.write_text("kernel v1\n")
    entry = {"bytes_per_launch": 123, "source_sha": bench.source_hash(str(src))}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k.cu": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k.cu") == 123
    src.write_text("kernel v2\n")                      # the kernel changed since the capture
    assert bench.dram_traffic("k.cu") is None
    assert bench.dram_traffic("other.cu") is None


def test_committed_traffic_entry_names_its_capture():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        table = json.load(f)
    for name, e in table.items():
        assert os.path.exists(os.path.join(bench.ROOT, e["capture"])), name
        assert e["bytes_per_launch"] > 0 and len(e["source_sha"]) == 16
