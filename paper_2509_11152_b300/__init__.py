"""B300-native strong recursive skeletonisation solver for symmetric H^2 matrices.

The compute path is the CUDA library ``libh2rs.so`` (sources in ``csrc/``, C-ABI in
``include/h2rs.h``); :mod:`.binding` is its thin ctypes binding.
"""
from .binding import (H2_PREC_FP32, H2_PREC_FP64, H2_PREC_TF32X3, H2Error, colmajor, h2_factor_create,
                      h2_factor_stats_get, h2_layout_get, h2_matrix_batch_info, h2_matrix_create,
                      h2_matrix_create_batch, h2_matvec, h2_matvec_static, h2_plan_query,
                      h2_plan_query_batch,
                      h2_refine_solve, h2_solve, h2_version, lib)

__all__ = ["H2_PREC_FP32", "H2_PREC_FP64", "H2_PREC_TF32X3", "H2Error", "colmajor", "h2_factor_create",
           "h2_factor_stats_get", "h2_layout_get", "h2_matrix_batch_info", "h2_matrix_create",
           "h2_matrix_create_batch", "h2_matvec", "h2_matvec_static", "h2_plan_query", "h2_plan_query_batch",
           "h2_refine_solve", "h2_solve", "h2_version", "lib"]
