"""The stored oracle results for the 1920x1080x200 workload
(tests/golden/cdmd_1080p_x200.json) are consistent with the oracle and the
input generator they claim to come from (CPU only).

* the clip the generator renders today has the stored per-frame sums (and,
  on the machine that wrote the file, the same SHA-256);
* row 0 of the stored sketch equals C_0 . D recomputed over all pixels
  (Algorithm 1 step 3), to FP64 summation-order rounding;
* the stored sigma are the leading stored singular values of Y, and the
  stored F-measures follow from their TP / FP / FN counts (Section 4);
* G has the shape (n-1) x r with finite entries, and the eigenvalues come in
  adjacent conjugate pairs with +Im first (the ordering reading).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import videogen
from oracle import measurement as M

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cdmd_1080p_x200.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def clip(gold):
    w = gold["workload"]
    return videogen.make_clip(w["width"], w["height"], w["n"], seed=w["clip_seed"], drift=w["drift"])


def test_clip_matches_stored_render(gold, clip):
    sums = clip.frames.sum(axis=1, dtype=np.int64)
    diff = int(np.abs(sums - np.array(gold["frame_sums"])).sum())
    assert diff <= 1e-7 * clip.frames.size * 128
    if diff == 0:
        assert hashlib.sha256(clip.frames.tobytes()).hexdigest() == gold["frames_sha256"]


def test_sketch_row_zero_recomputed(gold, clip):
    w = gold["workload"]
    assert gold["dy_rows"][0] == 0
    row = np.zeros(w["n"])
    for j0 in range(0, clip.m, 1 << 18):
        cols = np.arange(j0, min(clip.m, j0 + (1 << 18)))
        c0 = M.gaussian_block(w["c_seed"], [0], cols)[0]
        row += clip.frames[:, cols].astype(np.float64) @ c0
    ref = np.array(gold["dy"][0])
    assert np.max(np.abs(row - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_stored_quantities_are_consistent(gold):
    w = gold["workload"]
    r, n = w["r"], w["n"]
    sv = np.array(gold["y_singular_values"])
    np.testing.assert_allclose(np.array(gold["sigma"]), sv[:r], rtol=1e-12)
    assert np.all(np.diff(sv) <= 0)
    G = np.array(gold["G"])
    assert G.shape == (n - 1, r, 2) and np.all(np.isfinite(G))
    lam = np.array([complex(a, b) for a, b in gold["lam"]])
    i = 0
    while i < r:                                   # conjugate pairs adjacent, +Im first
        if abs(lam[i].imag) > 1e-9 * max(1.0, abs(lam[i])):
            assert lam[i].imag > 0 and i + 1 < r and abs(lam[i + 1] - np.conj(lam[i])) <= 1e-9 * abs(lam[i])
            i += 2
        else:
            i += 1
    for form in ("omp", "mlp"):
        g = gold[form]
        assert len(g["sel"]) == w["K"] and len(set(g["sel"])) == w["K"]
        p = g["tp"] / (g["tp"] + g["fp"])
        rc = g["tp"] / (g["tp"] + g["fn"])
        assert abs(g["F"] - 2 * p * rc / (p + rc)) <= 1e-15
        assert len(g["bg_samples"]) == gold["bg_sample_count"]
    assert gold["omp"]["tp"] + gold["omp"]["fn"] == gold["truth_count"]
