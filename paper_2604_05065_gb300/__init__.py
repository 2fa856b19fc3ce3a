"""GB300-native APLICUR: adaptive CUR-preconditioned LSQR for
min ||A x - b||^2 + mu ||x||^2 (Huh, Cartis, Nakatsukasa, arXiv 2604.05065).

The solver lives in the CUDA library libaplicur.so (C ABI in include/aplicur.h);
`aplicur` is its Python binding and `workloads` holds seeded synthetic inputs.
"""
from .aplicur import (AplicurError, BatchSolver, DeviceAllocator, Solver, aplicur_solve_fn, default_options, load,  # noqa
                      solve, launch_count, PREC_FP64, PREC_MIXED, PREC_DF32,
                      SKETCH_SPARSE_SIGN, SKETCH_GAUSSIAN, SKETCH_SRHT, PROFILE_FAMILIES)
