"""GB300 black-box randomized compression of HBS matrices (Levitt & Martinsson).

The computation lives in ``lib/libhbs.so`` (CUDA for sm_103a, C ABI in ``include/hbs.h``);
``paper_2205_02990_gb300.hbs`` is its thin Python binding. Build with
``python -m paper_2205_02990_gb300.build``.
"""

from .hbs import (factor_layout, hbs_apply_batch, hbs_autotune, hbs_get_tuning, hbs_load_factors,
                  hbs_set_graph, hbs_set_tuning,
                  HBS_PREC_FP64, HBS_PREC_FP64_TC, HBS_PREC_MIXED_BF16X3, HBS_PREC_MIXED_COMPENSATED, HBS_PREC_MIXED_BF16X6, Handle, HBSError, Problem, hbs_apply, hbs_apply_static, hbs_compress,
                  hbs_copy_factors, hbs_draw_gaussian, hbs_execute, hbs_factor_bytes, hbs_free,
                  hbs_get_node, hbs_plan, hbs_sample, hbs_sample_execute, hbs_sample_products, hbs_sample_sync, hbs_sync_status, hbs_tree, hbs_tree_build,
                  hbs_test_inject_status, hbs_probe_peaks, hbs_profile_sweep, hbs_probe_dmma,
                  hbs_probe_mma_issue, load)

__all__ = ["factor_layout", "hbs_apply_batch", "hbs_autotune", "hbs_get_tuning", "hbs_load_factors",
           "hbs_set_graph", "hbs_set_tuning", "HBS_PREC_FP64", "HBS_PREC_FP64_TC", "HBS_PREC_MIXED_BF16X3", "HBS_PREC_MIXED_COMPENSATED", "HBS_PREC_MIXED_BF16X6", "Handle", "HBSError", "Problem", "hbs_apply", "hbs_apply_static", "hbs_compress",
           "hbs_copy_factors", "hbs_draw_gaussian", "hbs_execute", "hbs_factor_bytes", "hbs_free",
           "hbs_get_node", "hbs_plan", "hbs_sample", "hbs_sample_execute", "hbs_sample_products", "hbs_sample_sync", "hbs_sync_status", "hbs_tree",
           "hbs_tree_build", "hbs_test_inject_status", "hbs_probe_peaks", "hbs_profile_sweep", "hbs_probe_dmma", "hbs_probe_mma_issue", "load"]
