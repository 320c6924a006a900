"""GB300-native spin-image generation with dynamic loop scheduling.

The compute path is libspin_gb300.so (CUDA for sm_103a, C ABI in
include/spin.h); this package is its thin Python binding (``si_*`` names, as
in C) plus seeded workload generators (``workloads``).
"""
from ._binding import (  # noqa: F401
    SCHED_NAMES, SI_ERR_BUSY, SI_ERR_CUDA, SI_ERR_INVALID, SI_ERR_OOM, SI_ERR_OVERFLOW, SI_ERR_TIMEOUT, SI_OK,
    SI_SCHED_AF, SI_SCHED_AWF, SI_SCHED_FAC, SI_SCHED_FAC_PROB, SI_SCHED_GSS, SI_SCHED_SS, SI_SCHED_STATIC, SI_BIN_BILINEAR, SI_BIN_NEAREST,
    BIN_NAMES, SpinError, batch_items, exported_names, load,
    make_schedule, si_candidate_rc2, si_candidate_rc2_binned, si_check_bounded_wait, si_match, SI_MATCH_FP32,
    SI_MATCH_BF16, si_chunk_table, si_schedule_chunks, si_default_workers, si_generate, si_generate_batched, si_generate_host,
    si_generate_noalloc, si_generate_probe, si_get_stats, si_last_error, si_mesh_create, si_mesh_destroy, si_mesh_prepare,
    si_reset_stats, si_serve_add_mesh, si_serve_create, si_serve_destroy, si_serve_poll, si_serve_release,
    si_serve_result, si_serve_submit, si_serve_wait, si_set_timing, si_tune_clear, si_tune_load, si_tune_lookup,
    si_tune_mesh, si_tune_save, si_version, si_kernel_launches, si_peak_smem_atomics, device_view,
    si_alloc_stats, si_debug_fail_allocs, si_generate_traced)
