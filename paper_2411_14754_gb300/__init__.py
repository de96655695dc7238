"""GB300-native SuCo (Subspace Collision) approximate nearest-neighbour search.

The query path runs in hand-written CUDA kernels for sm_103a behind the C ABI
of ``include/suco.h``; ``paper_2411_14754_gb300.suco`` is its Python binding.
"""
from .suco import (SucoError, SucoIndex, load_library, suco_autotune, suco_build_index, suco_build_index_from_assignments,  # noqa: F401
                   suco_build_index_from_parts,
                   suco_export_index, suco_free, suco_index_get_info, suco_kmeans_noalloc, suco_last_error, suco_query_batch,
                   suco_query_debug, suco_thresholds, suco_version, SucoMlp, suco_query_features,
                   suco_mlp_predict, suco_mlp_forward, suco_mlp_backward, suco_adamw_step, suco_add_reduced_copies, suco_read_status,
                   suco_inject_fault, suco_sc_linear, suco_sc_linear_workspace_size, FAULT_NONE, FAULT_ALLOC, FAULT_LAUNCH, FAULT_WAIT_TIMEOUT)
