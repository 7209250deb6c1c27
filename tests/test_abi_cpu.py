"""Host-only checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching a device."""
import ctypes
import re

import numpy as np

import pytest

import __graft_entry__
from paper_1404_3448_gb300 import build as lor_build
from paper_1404_3448_gb300 import lor as L

HEADER = lor_build.INCLUDE + "/lor.h"


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lor_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_path(lib):
    names = declared_functions()
    for must in ["lor_encode_concat", "lor_build_sa", "lor_build_sa_workspace_size", "lor_lcp",
                 "lor_longest_overlap", "lor_longest_overlap_workspace_size", "lor_rmq_build",
                 "lor_rmq_query", "lor_rmq_table_elems", "lor_device_status", "lor_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        s = L.lor_status_string(code)
        assert s and s != "unknown status"
    assert L.lor_status_string(-99) == "unknown status"


def test_workspace_queries_are_host_only(lib):
    assert L.lor_build_sa_workspace_size(0, 7) == 0
    prev = 0
    for n in [1, 2, 3, 10, 1000, 10**6]:
        w = L.lor_build_sa_workspace_size(n, 7)
        assert w >= prev and w % 256 == 0
        prev = w
    # under 64 bytes per symbol at scale (sort buffers + per-level arrays)
    assert L.lor_build_sa_workspace_size(10**8, 7) < 64 * 10**8
    assert L.lor_longest_overlap_workspace_size(1000) > 0
    assert L.lor_rmq_row_stride(1) == 64 and L.lor_rmq_row_stride(64) == 64
    assert L.lor_rmq_row_stride(65) == 128
    assert L.lor_rmq_table_elems(1) == 64
    assert L.lor_rmq_table_elems(8) == 4 * 64
    assert L.lor_rmq_table_elems(1 << 20) == 21 * (1 << 20)
    assert L.lor_radix_sort_workspace_size(0) > 0


def test_bad_arguments_rejected_on_host(lib):
    assert L.lor_build_sa(None, 10, 7, None, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_build_sa(1 << 20, 0, 7, 1 << 20, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_build_sa(1 << 20, 10, 1, 1 << 20, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_build_sa(1 << 20, 1 << 40, 7, 1 << 20, None, 0, None) == L.LOR_ERR_TOO_LARGE
    assert L.lor_build_sa(1 << 20, 10, 7, 1 << 20, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert L.lor_build_sa(1 << 20, 10, 7, 1 << 20, (1 << 20) + 8, 1 << 30, None) == L.LOR_ERR_WORKSPACE
    assert L.lor_lcp(None, None, 5, None, None, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_lcp(256, 256, 5, 256, 256, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert L.lor_lcp_workspace_size(1000) >= 24 * 1000
    assert L.lor_longest_overlap(1, 1, 5, 1, 0, 1, None, 0, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_longest_overlap(1, 1, 5, 1, 251, 1, None, 0, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_longest_overlap(256, 256, 5, 256, 2, 256, None, 4, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_longest_overlap(256, 256, 5, 256, 2, 256, None, 0, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert L.lor_rmq_build(None, 5, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_rmq_build(256, 5, 256, 4, None) == L.LOR_ERR_WORKSPACE
    assert L.lor_rmq_build(256, 5, 256 + 4, 1 << 10, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_rmq_query(None, None, 5, None, None, 1, None, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_rmq_query(256, 256, 5, None, None, 0, None, None) == L.LOR_OK
    lens = (ctypes.c_int64 * 2)(3, 4)
    assert L.lor_encode_concat(256, lens, 0, 256, None, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_encode_concat(256, lens, 251, 256, None, None) == L.LOR_ERR_INVALID_ARG
    neg = (ctypes.c_int64 * 2)(3, -1)
    assert L.lor_encode_concat(256, neg, 2, 256, None, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_radix_sort_pairs(None, None, 5, 8, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert L.lor_radix_sort_pairs(None, None, 0, 8, None, 0, None) == L.LOR_OK
    assert L.lor_radix_sort_pairs(256, 256, 5, 65, None, 0, None) == L.LOR_ERR_INVALID_ARG


def test_no_oracle_in_product_path():
    import os
    pkg = os.path.dirname(lor_build.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "lor_oracle" not in txt, f


def test_server_batch_bytes_host_only(lib):
    work1, res1 = L.server_batch_bytes([1000, 2000])
    assert work1 > 0 and res1 > 0
    # one pair: workspace covers the grouped pipeline (text 3002 symbols) plus
    # input, records and positions; resident = ISA + LCP + the block table over
    # ceil(3002 / 32) = 94 block minima, with bit_width(3002 // 32) = 7 rows of
    # 128 entries (linear space, far below a full sparse table's 12 rows of n)
    n = 3002
    assert res1 >= 4 * n + 4 * n + 4 * 7 * 128
    assert res1 < 4 * n + 4 * 12 * n
    assert work1 >= L.lor_batch_workspace_size(np.array([1000, 2000], np.int64).ctypes.data, 1)
    work2, res2 = L.server_batch_bytes([1000, 2000, 5, 7])
    assert work2 >= work1 and res2 >= res1
    # more pairs than one group holds, negative lengths: rejected
    assert L.server_batch_bytes([10] * 1026) == (0, 0)
    assert L.server_batch_bytes([10, -1]) == (0, 0)


def test_server_config_validation_is_host_only(lib):
    bad = [
        L.ServerConfig(1 << 30, 0, 8, 1 << 20),    # no workers
        L.ServerConfig(1 << 30, 9, 8, 1 << 20),    # too many workers
        L.ServerConfig(1 << 30, 2, 513, 1 << 20),  # more pairs than one group holds
        L.ServerConfig(1 << 30, 2, 8, 0),
        L.ServerConfig(1 << 30, 2, 8, (1 << 28) + 1),
        L.ServerConfig(1000, 2, 8, 1 << 20),       # below one granule
    ]
    for cfg in bad:
        h = ctypes.c_void_p()
        assert lib.lor_server_create(ctypes.byref(cfg), ctypes.byref(h)) == L.LOR_ERR_INVALID_ARG
        assert not h.value
    assert lib.lor_server_create(None, None) == L.LOR_ERR_INVALID_ARG
    for fn, args in [("lor_server_poll", (None, None, 1, 0)), ("lor_server_release", (None, 1)),
                     ("lor_server_stats_get", (None, None)), ("lor_server_destroy", (None,)),
                     ("lor_server_query", (None, 1, None, None, 1, None))]:
        assert getattr(lib, fn)(*args) == L.LOR_ERR_INVALID_ARG


@pytest.mark.skipif(L.torch.cuda.is_available(), reason="checks the no-device path")
def test_server_create_without_device_fails_cleanly(lib):
    cfg = L.ServerConfig(1 << 26, 1, 8, 1 << 20)
    h = ctypes.c_void_p()
    assert lib.lor_server_create(ctypes.byref(cfg), ctypes.byref(h)) == L.LOR_ERR_CUDA
    assert not h.value


def test_batch_graph_workspace_covers_the_batch_workspace(lib):
    lens = np.array([1000, 2000, 0, 5, 300000, 1], dtype=np.int64)
    base = L.lor_batch_workspace_size(lens.ctypes.data, 3)
    g = L.lor_batch_graph_workspace_size(lens.ctypes.data, 3)
    assert base > 0 and g > base and g % 256 == 0
    assert L.lor_batch_graph_workspace_size(lens.ctypes.data, 0) == 0
    h = ctypes.c_void_p()
    # bad arguments are refused on the host, before any capture
    assert L.lor_batch_graph_create(None, lens.ctypes.data, 0, None, None, None, 0, None, 0,
                                    ctypes.byref(h)) == -1
    assert L.lor_batch_graph_launch(None, None) == -1
    assert L.lor_batch_graph_destroy(None) == 0


def test_tune_configuration_round_trip_and_range_checks(lib):
    import paper_1404_3448_gb300 as P
    d = P.tune_default()
    assert d == {"digit_bits": 8, "level0_key_bits": 48, "sort_items_64": 12, "sort_items_32": 16,
                 "merge_items": 4}
    try:
        assert P.tune_set(digit_bits=6, merge_items=8)["digit_bits"] == 6
        assert P.tune_get()["merge_items"] == 8
        for bad in [dict(digit_bits=4), dict(digit_bits=9), dict(level0_key_bits=23),
                    dict(level0_key_bits=61), dict(sort_items_64=20), dict(sort_items_32=8),
                    dict(merge_items=3), dict(merge_items=16)]:
            before = P.tune_get()
            with pytest.raises(L.LorError):
                P.tune_set(**bad)
            assert P.tune_get() == before  # a refused value changes nothing
    finally:
        P.tune_set(**d)
    assert P.tune_get() == d


def test_int64_path_host_checks(lib):
    """The *64 calls: sizes past the int32 range are accepted up to LOR_MAX_N64,
    bad arguments are rejected before any device access."""
    n32, n64 = L.LOR_MAX_N, L.LOR_MAX_N64
    assert n64 > 2**31 and n64 < 2**32
    # workspace queries: host only, monotone, zero outside [1, LOR_MAX_N64]
    assert lib.lor_build_sa64_workspace_size(0, 7) == 0
    assert lib.lor_build_sa64_workspace_size(n64 + 1, 7) == 0
    assert lib.lor_build_sa64_workspace_size(1000, 1) == 0
    big = lib.lor_build_sa64_workspace_size(n32 + 1, 7)
    assert big > 0 and big % 256 == 0 and big < 48 * (n32 + 1)
    assert lib.lor_lcp64_workspace_size(n64) > 0 and lib.lor_lcp64_workspace_size(n64 + 1) == 0
    assert lib.lor_longest_overlap64_workspace_size(n32 + 1) > 0
    assert L.lor_build_sa_workspace_size(n32 + 1, 7) == 0  # the int32 call stops at LOR_MAX_N
    assert lib.lor_rmq_block_table_elems(n32 + 1) > 0  # the block table serves both paths
    prev = 0
    for n in [1, 2, 3, 10, 1000, 10**6]:
        w = lib.lor_build_sa64_workspace_size(n, 7)
        assert w >= prev
        prev = w
    # argument checks
    assert lib.lor_build_sa64(None, 10, 7, None, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_build_sa64(256, 10, 1, 256, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_build_sa64(256, n64 + 1, 7, 256, None, 0, None) == L.LOR_ERR_TOO_LARGE
    assert lib.lor_build_sa64(256, 10, 7, 256, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert lib.lor_build_sa64(256, 10, 7, 256, 256 + 8, 1 << 30, None) == L.LOR_ERR_WORKSPACE
    assert lib.lor_lcp64(None, None, 5, None, None, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_lcp64(256, 256, n64 + 1, 256, 256, None, 0, None) == L.LOR_ERR_TOO_LARGE
    assert lib.lor_lcp64(256, 256, 5, 256, 256, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert lib.lor_longest_overlap64(256, 256, 5, 256, 0, 256, None, 0, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_longest_overlap64(256, 256, 5, 256, 2, 256, None, 4, None, 0, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_longest_overlap64(256, 256, n64 + 1, 256, 2, 256, None, 0, None, 0, None) == L.LOR_ERR_TOO_LARGE
    assert lib.lor_longest_overlap64(256, 256, 5, 256, 2, 256, None, 0, None, 0, None) == L.LOR_ERR_WORKSPACE
    assert lib.lor_rmq_block_query64(None, None, None, 5, None, None, 1, None, None) == L.LOR_ERR_INVALID_ARG
    assert lib.lor_rmq_block_query64(256, 256, 256, 5, None, None, 0, None, None) == L.LOR_OK
    assert lib.lor_rmq_block_query64(256, 256, 256, n64 + 1, 256, 256, 1, 256, None) == L.LOR_ERR_TOO_LARGE
    lens = (ctypes.c_int64 * 2)(3, 4)
    assert lib.lor_encode_concat64(256, lens, 0, 256, None, None) == L.LOR_ERR_INVALID_ARG
    huge = (ctypes.c_int64 * 2)(n64, 4)
    assert lib.lor_encode_concat64(256, huge, 2, 256, None, None) == L.LOR_ERR_TOO_LARGE
