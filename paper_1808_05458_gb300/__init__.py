"""GB300-native exact global minimum cut.

Method of Henzinger, Noe and Schulz, "Shared-memory Exact Minimum Cuts":
label-propagation / degree upper bound, Padberg-Rinaldi tests, concurrent
capped CAPFOREST scans and graph contraction, repeated until one vertex is
left -- as hand-written CUDA for sm_103a behind the C ABI in include/mc.h.

Python side: :mod:`paper_1808_05458_gb300.mincut` (ctypes binding).
"""
from .mincut import (MC_BOUND_BEST, MC_BOUND_DEGREE, MC_BOUND_LEARNED, MC_BOUND_LP, MC_EINVAL,
                     MC_ENOMEM, MC_EOVERFLOW, MC_OK, MC_PQ_FIFO, MC_PQ_LIFO, PROPOSER_PARAMS, Graph, MinCut,
                     MinCutError, Proposer,
                     batch_autotune, batch_min_cut, batch_set_shape, batch_shape_count, bitmap_to_side, load_library, min_cut,
                     options, strerror, test_fail_alloc_after)

__all__ = ["Graph", "MinCut", "MinCutError", "min_cut", "batch_min_cut", "batch_autotune",
           "batch_set_shape", "batch_shape_count",
           "options", "strerror", "Proposer", "PROPOSER_PARAMS", "MC_BOUND_LEARNED",
           "MC_BOUND_BEST",
           "load_library", "bitmap_to_side", "MC_PQ_LIFO", "MC_PQ_FIFO", "MC_BOUND_DEGREE",
           "MC_BOUND_LP", "MC_OK", "MC_EINVAL", "MC_EOVERFLOW", "MC_ENOMEM",
           "test_fail_alloc_after"]
