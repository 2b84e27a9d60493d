"""GB300-native randomized GENP (Pan & Qian, arXiv:1212.4560, Sec. 1.1).

Solve A x = b by Gaussian elimination with no pivoting on C = A G for a
random multiplier G, returning x = G y from L U y = b, with FP64 iterative
refinement.  The arithmetic runs in the CUDA library libgenp.so (C ABI in
include/genp.h); this package only marshals arguments.
"""
from ._lib import (BF16, BF16_SLICED, BF16X3, CIRCULANT, CIRCULANT_PM1, FP8_E4M3, FP32, FP64,  # noqa: F401
                   GAUSSIAN, HOUSEHOLDER_PM1, IDENTITY, LEFT, RIGHT, SPARSE_PM1, STATUS_NAMES, TOEPLITZ, GenpError)
from .api import (Factors, Info, Multiplier, adjoint, block_factor, factor, info_fetch, launch_count, lowrank,  # noqa: F401
                  numerical_rank,
                  make_multiplier, multiplier_export, precondition, redraw_multiplier, refactor, refine, solve,
                  solve_system, status_string, version)
