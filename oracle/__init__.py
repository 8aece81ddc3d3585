"""FP64 CPU oracle for compressed DMD background modelling.

TEST INFRASTRUCTURE.  A plain, slow, obviously-correct implementation of what
the CUDA path computes, written from the paper (Erichson, Brunton & Kutz,
"Compressed Dynamic Mode Decomposition for Background Modeling",
arXiv 1512.04205).  It shares no code with the CUDA path and neither imports
the other.  Only `tests/`, the smoke check and the benchmark's CPU-baseline
leg may import it; the product path never routes through it.

Modules
  philox       Philox4x32-10 (Salmon et al., SC'11), numpy uint64 arithmetic
  measurement  Gaussian / Rademacher / sparse / single-pixel C (Section 3.3)
  cdmd         Algorithm 1, OMP (Remark 3), background, mask, F-measure
"""
from . import philox, measurement, cdmd  # noqa: F401
