"""GB300 (sm_103a) EGLM-MHD block-pool step of the MAP method (arXiv:1204.5849).

The compute path is libmapgb300.so (hand-written CUDA kernels behind the C ABI in
include/map.h); this package holds its sources (csrc/), the in-tree build (_build.py)
and a thin ctypes binding (binding.py).
"""

from .binding import (MAP_FP32_FIX64, MAP_FP64, MapError, Partition, Pool, check_leaves, exported_symbols,
                      load, make_params, make_refine, plan_leaves, plan_partition)
from .autotune import choose_block_size

__all__ = ["Pool", "MapError", "MAP_FP64", "MAP_FP32_FIX64", "load", "exported_symbols",
           "make_params", "make_refine", "choose_block_size", "check_leaves", "plan_leaves", "Partition",
           "plan_partition"]
