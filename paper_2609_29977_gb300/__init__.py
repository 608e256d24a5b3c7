"""GB300-native direct solver for the SPD root-coupled KKT systems of branch
MPC (two-level parallel Cholesky, Alg. 1, and triangular solves, Alg. 2).

The compute runs in the CUDA library ``libbm.so`` (C ABI in include/bm.h);
``paper_2609_29977_gb300.bm`` is its thin ctypes binding. Importing the
package does not load the library; the first call does, and raises if the
library was not built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from .bm import (BATCH_NB, BranchKKTBatch, bm_batch_analyze, bm_batch_destroy, bm_batch_factor, bm_batch_query,
                 bm_batch_schedule, bm_batch_solve, bm_batch_workspace_bytes)
from .bm import bm_assemble_reduced, bm_test_bounded_wait
from .bm import (BM_REQ_HOST_IO, BM_SERVE_MAX_RHS, BranchKKTServer, bm_server_create, bm_server_destroy,
                 bm_server_get_stats, bm_server_poll, bm_server_request_bytes, bm_server_submit, make_server_desc)
from .bm import (BM_FLAG_COUPLING_FP32, BM_FLAG_COUPLING_REFINE, BM_FLAG_NO_GRAPH, BM_FLAG_NO_TUNE, BM_FLAG_RESIDUAL_FP64, BM_PREC_FP32_IR, bm_residual, ff_residual, BM_PREC_FP64, BMError, BranchKKTSolver, bm_analyze,
                 bm_destroy, bm_export_factor, bm_factor, bm_factor_solve_host, bm_factor_solve_noalloc, bm_query, bm_round_to_fp32, bm_schedule, bm_solve,
                 bm_status_string, bm_version, bm_workspace_bytes, library_path)

__all__ = ["BranchKKTBatch", "BATCH_NB", "bm_batch_analyze", "bm_batch_factor", "bm_batch_solve", "bm_batch_query",
           "bm_batch_schedule", "bm_batch_destroy", "bm_batch_workspace_bytes", "BranchKKTSolver", "BMError", "bm_analyze", "bm_factor", "bm_solve", "bm_query",
           "bm_export_factor", "bm_factor_solve_host", "bm_factor_solve_noalloc", "bm_round_to_fp32", "bm_destroy", "bm_workspace_bytes",
           "bm_version", "bm_status_string", "library_path", "BM_PREC_FP64", "BM_PREC_FP32_IR",
           "BM_FLAG_NO_GRAPH", "BM_FLAG_COUPLING_REFINE", "BM_FLAG_COUPLING_FP32", "BM_FLAG_NO_TUNE", "BM_FLAG_RESIDUAL_FP64", "bm_residual", "ff_residual", "bm_schedule", "BranchKKTServer", "BM_REQ_HOST_IO", "BM_SERVE_MAX_RHS", "bm_server_create",
           "bm_server_destroy", "bm_server_get_stats", "bm_server_poll", "bm_server_request_bytes",
           "bm_server_submit", "make_server_desc", "bm_assemble_reduced", "bm_test_bounded_wait"]
