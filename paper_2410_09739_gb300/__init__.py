"""GB300 (sm_103a) implementation of the D3Q27 Fokker-Planck central-moment LBM.

The compute path is libfpclbm.so (CUDA kernels behind the C ABI of
include/fpclbm.h); ``fpclbm`` is its thin ctypes binding.  Importing this
package does not load the library; the first call does, and raises if it has
not been built (there is no CPU fallback).
"""
from .fpclbm import (  # noqa: F401
    FPCLBM_BC_PERIODIC, FPCLBM_BC_WALLS_Y, FPCLBM_DIFF_EQUILIBRIUM, FPCLBM_DIFF_FP, FPCLBM_DIFF_FP_LEARNED,
    FPCLBM_FP32, FPCLBM_FP32_STORE_BF16, FPCLBM_FP32_STORE_FP16, FPCLBM_FP64, FpclbmError, Lattice, load,
)
