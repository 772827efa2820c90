"""GB300-native compressed 3D FFL-MPI reconstruction (arXiv 2511.06627).

The hot path -- the compressed forward operator A, its adjoint and the
regularised accelerated projected-gradient solve -- runs in hand-written
sm_103a CUDA kernels behind the C ABI of include/mpi_ffl.h (libmpiffl.so).
This package is the thin Python binding over that ABI.
"""

from . import _lib  # noqa: F401
from ._lib import (  # noqa: F401
    PATH_FULL_GEMM,
    PATH_FUSED,
    PATH_LINE_GEMM,
    PATH_STAGED,
    PATHS,
    PREC_BF16X3,
    PREC_FP32,
    PREC_TF32,
    STAGE_EVB,
    STAGE_F,
    STAGE_H,
    STAGE_P,
    MpiFflError,
)


def __getattr__(name):
    # torch-facing classes are imported on first use, so that `build()` and the
    # CPU-side symbol checks need neither a GPU nor a CUDA-enabled torch
    if name == "FFLOperator":
        from .operator import FFLOperator

        return FFLOperator
    raise AttributeError(name)
