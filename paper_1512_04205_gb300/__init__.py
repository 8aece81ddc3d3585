"""GB300-native compressed DMD (cDMD) for video background modelling.

The compute path lives in libcdmd.so (CUDA kernels for sm_103a behind the C
ABI of include/cdmd.h); `cdmd` is its thin Python binding.  Build with
`python -m paper_1512_04205_gb300.build`.
"""
from . import cdmd  # noqa: F401
from .cdmd import (CdmdError, Context, Measure, cdmd_decompose, cdmd_lift,  # noqa: F401
                   cdmd_run, cdmd_run_host, cdmd_sketch, cdmd_sketch_gather,
                   cdmd_status_sync, cdmd_subtract, load_library, make_params,
                   unpack_mask)
