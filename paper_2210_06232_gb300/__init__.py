"""GB300-native exponential-integrator Fourier pseudospectral solver for the
periodic 3D Maxwell equations (Wang & Jiang, arXiv 2210.06232).

The compute path is the C-ABI library ``lib/libmaxexp.so`` (hand-written
sm_103a CUDA; declared in ``include/maxexp.h``); ``maxexp`` is its ctypes
binding.  Build it with ``python paper_2210_06232_gb300/build.py``.
"""
from .maxexp import (  # noqa: F401
    MX_FORM_LITERAL,
    MX_FORM_SPECTRAL,
    MX_FORM_XY,
    MX_FP32,
    MX_FP64,
    MaxexpError,
    Solver,
    footprint_bytes,
)
