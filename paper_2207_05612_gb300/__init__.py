"""dmrgc: GB300-native circuit-DMRG compression sweep (arXiv:2207.05612).

The compute lives in libdmrgc.so (CUDA, sm_103a); `binding` is its ctypes
binding.  Build with `python -m paper_2207_05612_gb300.build`.
"""
from .binding import (DMRGC_BF16X3, DMRGC_FP32, DMRGC_FP64, DMRGC_TF32X3, Context,  # noqa: F401
                      DmrgcError, lib)
