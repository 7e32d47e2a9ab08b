"""GB300 (sm_103a) cell-based FMM gravity solve (Octo-Tiger, arXiv 1908.03121).

The solve lives in the CUDA library built from ``csrc/`` (C ABI:
``include/fmm_gb300.h``); ``fmm`` is its Python binding.
"""

from .fmm import (FmmError, Solver, Tree, fmm_build_tree, fmm_get_sizes, fmm_get_stats,
                  fmm_upward, fmm_m2l, fmm_downward, fmm_forces, fmm_step, fmm_set_tuning,
                  fmm_get_tuning, fmm_forces_noalloc, fmm_check_conversions, fmm_peak_rate,
                  fmm_scf_update, scf_params, fmm_field_time_derivative, fmm_get_status,
                  fmm_destroy_tree, fmm_last_error, load, library_path, FMM_FP64, FMM_MIXED,
                  FMM_DFLOAT, FMM_STATUS_BAD_DENSITY)

__all__ = ["FmmError", "Solver", "Tree", "fmm_build_tree", "fmm_get_sizes", "fmm_get_stats",
           "fmm_upward", "fmm_m2l", "fmm_downward", "fmm_forces", "fmm_step", "fmm_set_tuning",
           "fmm_get_tuning", "fmm_forces_noalloc", "fmm_check_conversions", "fmm_peak_rate",
           "fmm_scf_update", "scf_params", "fmm_field_time_derivative",
           "fmm_get_status",
           "fmm_destroy_tree", "fmm_last_error", "load", "library_path", "FMM_FP64", "FMM_MIXED",
           "FMM_DFLOAT", "FMM_STATUS_BAD_DENSITY"]
