"""GB300-native sparse Fast Chebyshev Transform (hot path behind a C ABI).

The transform runs in libfct_gb300.so (hand-written CUDA for sm_103a); the
modules here only build that library and marshal arguments to it.
"""
from .fct import (FCT_FAMILY_GAUSSCOS, FCT_FAMILY_POLY, FCT_FAMILY_POLY_GAUSSCOS, FCT_FAMILY_RATIONAL,  # noqa: F401
                  FCT_FP64, FCT_GRID_EXTREMA, FCT_GRID_FIRST_KIND, FCT_MIXED, FCT_PLAN_BUILD_AUTO,
                  FCT_PLAN_BUILD_DEVICE, FCT_PLAN_BUILD_HOST, FctError, Plan, fct_alias_tables_host, fct_batch_create,
                  fct_batch_destroy, fct_batch_launch, fct_batch_reports,
                  fct_default_options, fct_destroy, fct_evaluate, fct_execute, fct_execute_batch, fct_execute_host,
                  fct_execute_noalloc, fct_grid_offsets, fct_measure_fp64, fct_measure_l2, fct_measure_team_barrier,
                  fct_plan_apply, fct_plan_clone, fct_plan_condition, fct_plan_create, fct_plan_get_info,
                  fct_plan_last_report, fct_plan_rhs, fct_plan_tables, fct_sample, fct_server_create,
                  fct_server_destroy, fct_server_poll, fct_server_submit, fct_server_wait, lib, library_path)
