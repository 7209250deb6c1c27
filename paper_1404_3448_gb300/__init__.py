"""GB300-native longest-overlap-region library (arXiv 1404.3448).

DC3 suffix array, Kasai LCP, cross-sequence max-LCP overlap and sparse-table
RMQ as hand-written CUDA kernels for sm_103a behind the C ABI in
include/lor.h; ``lor`` is the thin Python binding.
"""
from . import build  # noqa: F401
from .lor import (  # noqa: F401
    Batch, BatchGraph, LorError, Pipeline, Server, build_sa, check_device, device_status, encode_concat, last_dc3_trace,
    lcp, load, longest_overlap, overlap_dict, profile_enable, profile_read, profile_reset,
    radix_sort_pairs, rmq_build, rmq_query, rmq_block_build, rmq_block_query, rmq_block_argmin, server_batch_bytes, workspace, tune_default, tune_get, tune_set,
    autotune_batch, multi_query_overlap, topk_overlaps,
    encode_concat64, build_sa64, lcp64, longest_overlap64, overlap64_dict, rmq_block_query64,
    dc3_route, dc3_route_get, dc3_route_set, test_set_wait, status_string,
    LOR_OK, LOR_ERR_BAD_SYMBOL, LOR_ERR_TIMEOUT, LOR_ERR_INVALID_ARG,
)
