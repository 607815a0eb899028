"""GB300-native incidence-constrained multilevel hypergraph partitioning.

The library (libhgp.so, C ABI in include/hgp.h) runs the whole data-parallel
path of arXiv 2604.14411 in hand-written CUDA kernels for sm_103a; this
package holds its sources, its build step and a thin ctypes binding.
"""
from .hgp import (EXPORTS, HGP_DEBUG_KEEP_LEVELS, HGP_DEBUG_TIMING, Graph, HgpError, Model,
                  Result, hgp_create, hgp_destroy, hgp_error_string, hgp_get_level_array,
                  hgp_get_stats, hgp_last_error, hgp_model_from_params, hgp_partition,
                  hgp_partition_batch, hgp_train_mlp, load, train_model)

__all__ = ["Graph", "HgpError", "Result", "EXPORTS", "load", "hgp_create", "hgp_partition",
           "hgp_get_stats", "hgp_get_level_array", "hgp_error_string", "hgp_last_error",
           "hgp_destroy", "HGP_DEBUG_KEEP_LEVELS", "HGP_DEBUG_TIMING", "Model",
           "hgp_partition_batch", "hgp_train_mlp", "hgp_model_from_params", "train_model"]
