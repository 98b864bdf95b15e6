"""GB300-native fused generate-and-sketch library (arXiv 2603.20966).

Y = S A (left) and Y = A S^T (right) with S a dense Gaussian / Rademacher /
uniform matrix regenerated tile by tile from Philox4x32-10 inside the
kernels.  The compute path is ``libsketch.so`` (hand-written CUDA for
sm_103a) behind the C ABI in ``include/sketch.h``; this package is its thin
Python binding plus a small convenience class over torch tensors.
"""
from __future__ import annotations

from ._native import (SK_BF16X2, sk_batch_add, sk_batch_create, sk_batch_destroy,
                      sk_batch_run, sk_batch_size, sk_batch_status, sk_batch_tune, SK_FP8E4M3, SK_FP32, SK_GAUSSIAN, SK_RADEMACHER, SK_UNIFORM,
                      SketchError, sk_apply_left, sk_apply_left_host, sk_apply_right,
                      sk_apply_right_host, sk_create, sk_debug_set_wait, sk_debug_status, sk_destroy, sk_get_info, sk_launch_count, sk_materialize,
                      sk_profile_events,
                      sk_set_precision, sk_set_workspace, sk_stream_status, sk_version,
                      sk_workspace_size, status_string)
from ._native import (sk_apply_left_noalloc, sk_apply_left_stored, sk_apply_right_e4m3,
                      sk_batch_config, sk_batch_set_config, sk_nystrom, sk_quantize_e4m3)
from ._native import (sk_server_create, sk_server_destroy, sk_server_fetch, sk_server_poll,
                      sk_server_release, sk_server_reset_stats, sk_server_stats_get,
                      sk_server_submit, sk_server_wait)
from .sketch import Server, Sketch

__all__ = [
    "Sketch", "SketchError", "SK_GAUSSIAN", "SK_RADEMACHER", "SK_UNIFORM", "SK_FP32", "SK_BF16X2",
    "SK_FP8E4M3", "sk_create", "sk_set_precision", "sk_get_info", "sk_apply_left",
    "sk_apply_right", "sk_apply_left_host", "sk_apply_right_host", "sk_materialize",
    "sk_workspace_size", "sk_set_workspace", "sk_stream_status", "sk_debug_status",
    "sk_debug_set_wait", "sk_destroy", "sk_version", "sk_profile_events", "sk_launch_count",
    "status_string", "sk_batch_create", "sk_batch_add", "sk_batch_run", "sk_batch_tune",
    "sk_batch_status", "sk_batch_size", "sk_batch_destroy", "Server", "sk_server_create",
    "sk_server_submit", "sk_server_poll", "sk_server_wait", "sk_server_fetch",
    "sk_server_release", "sk_server_stats_get", "sk_server_reset_stats", "sk_server_destroy",
    "sk_quantize_e4m3", "sk_apply_right_e4m3", "sk_nystrom", "sk_apply_left_noalloc",
    "sk_apply_left_stored", "sk_batch_set_config", "sk_batch_config",
]
