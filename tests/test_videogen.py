"""The input generator's truth-from-spec helper returns what make_clip
returns as ground truth (CPU only)."""
import numpy as np
import pytest

import videogen


@pytest.mark.parametrize("w,h,n,seed,gen", [(160, 120, 30, 5, dict(drift=0.1)), (97, 61, 12, 8, dict(n_objects=8, shape="ellipse"))])
def test_truth_from_spec_matches_make_clip(w, h, n, seed, gen):
    clip = videogen.make_clip(w, h, n, seed=seed, **gen)
    spec = videogen.clip_spec(w, h, n, seed, **gen)
    assert np.array_equal(videogen.truth_from_spec(spec), clip.truth)
