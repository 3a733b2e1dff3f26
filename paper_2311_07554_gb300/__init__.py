"""GB300 (sm_103a) engine for sketch-based influence maximisation under the IC model.

The hot path (hash-sampled live-edge sketches, batched union-find connectivity, component
histograms and gains, compact sketches, device lazy greedy, spread) runs in hand-written
CUDA kernels behind the C ABI of ``include/im_gb300.h``; this package is its binding.
"""
from ._native import (  # noqa: F401
    IM_ECUDA, IM_EDEVICE, IM_EINVAL, IM_ENOMEM, IM_ESTATE, IM_ETIMEOUT, IM_HUBS_AUTO, IM_OK, IM_PROBS_ARRAY, IM_PROBS_UNIFORM, IM_PROBS_WIC,
    IM_PTR_DEVICE, IM_PTR_HOST, Batch, IMContext, IMServer, Mailbox, im_batch_schedule, im_batch_tune,
    IMError, im_autotune, im_footprint_estimate, im_build_sketches, im_create, im_destroy, im_get_centers, im_get_compact,
    im_get_gains, im_get_labels, im_hash_peak, im_load_graph, im_mc_spread, im_set_edge_probs, im_get_round_evals, im_get_stats, im_profile_enable,
    im_profile_get, im_profile_reset, im_reset_selection, im_run_batch, im_select_seeds,
    im_set_graph, im_set_hubs, im_set_pipeline, im_debug_fail_alloc, im_debug_record_cap, im_set_union_path, IM_UNION_FUSED, IM_UNION_RECORDS, IM_UNION_BUCKETS, IM_UNION_AUTO, im_set_seed_speculation, im_set_refresh_threshold, im_set_sketch_batch, im_sketch_static, im_spread, im_stream, lib)

__all__ = [n for n in dir() if n.startswith("im_")] + ["Batch", "IMContext", "IMServer", "IMError", "Mailbox", "lib"]
