"""GB300-native BLF-LS: bilateral filter embedded in least squares (arXiv 1812.07122).

The compute lives in ``libblfls.so`` (hand-written sm_103a CUDA kernels behind a C ABI, declared
in ``include/blfls.h``); :mod:`.blfls` is its thin ctypes binding and :mod:`.synth` makes seeded
synthetic inputs.  Importing the package does not load the library; the first binding call does,
and raises if it has not been built.
"""
from . import blfls  # noqa: F401
from .blfls import (  # noqa: F401
    BLFLS_BF16W,
    BLFLS_DETAIL_ENHANCE,
    BLFLS_FP16W,
    BLFLS_FP32,
    BLFLS_LOG_TONE,
    BlflsError,
    Smoother,
    blfls_blf_residual,
    blfls_create,
    blfls_destroy,
    blfls_gaussian,
    blfls_last_error,
    blfls_layers,
    blfls_smooth,
    blfls_smooth_batch,
    blfls_smooth_grid,
    blfls_smooth_guided,
    blfls_smooth_host,
    blfls_smooth_ls,
    blfls_smooth_nc,
    blfls_smooth_normalized,
    blfls_smooth_rolling,
    blfls_solve_residual,
    make_job,
)
