"""Thin Python binding of liblor (include/lor.h).

The ``lor_*`` functions take raw integers for device pointers and streams and
return the C status; the lower-case helpers below marshal torch tensors
(device memory, streams) into those calls and raise ``LorError`` on a
non-zero status.  Every step of the path runs in the library's CUDA kernels;
this module only allocates outputs and workspaces with torch and passes
pointers.  It raises ImportError when the compiled library is missing --
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

LOR_OK = 0
LOR_ERR_INVALID_ARG = -1
LOR_ERR_BAD_SYMBOL = -2
LOR_ERR_TOO_LARGE = -3
LOR_ERR_WORKSPACE = -4
LOR_ERR_CUDA = -5
LOR_ERR_TIMEOUT = -6
LOR_ERR_BAD_INPUT = -7
LOR_ERR_CANCELLED = -8
LOR_MAX_SEQ = 250

OVERLAP_FIELDS = ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b", "n_pos", "reserved")
LOR_MAX_N = 2147483000
LOR_MAX_N64 = 4294901760

_lib = None


class LorError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblor.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"liblor.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "lor_encode_concat": ([vp, vp, i32, vp, vp, vp], ctypes.c_int),
        "lor_build_sa_workspace_size": ([i64, i32], sz),
        "lor_build_sa": ([vp, i64, i32, vp, vp, sz, vp], ctypes.c_int),
        "lor_build_sa_noalloc": ([vp, i64, i32, vp, vp], ctypes.c_int),
        "lor_lcp_workspace_size": ([i64], sz),
        "lor_lcp": ([vp, vp, i64, vp, vp, vp, sz, vp], ctypes.c_int),
        "lor_longest_overlap_workspace_size": ([i64], sz),
        "lor_longest_overlap": ([vp, vp, i64, vp, i32, vp, vp, i64, vp, sz, vp], ctypes.c_int),
        "lor_batch_workspace_size": ([vp, i32], sz),
        "lor_batch_overlap": ([vp, vp, i32, vp, vp, vp, i64, vp, sz, vp], ctypes.c_int),
        "lor_batch_graph_workspace_size": ([vp, i32], sz),
        "lor_batch_graph_create": ([vp, vp, i32, vp, vp, vp, i64, vp, sz, vp], ctypes.c_int),
        "lor_batch_graph_launch": ([vp, vp], ctypes.c_int),
        "lor_batch_graph_kernels": ([vp], i64),
        "lor_batch_graph_destroy": ([vp], ctypes.c_int),
        "lor_topk_overlaps_workspace_size": ([i64], sz),
        "lor_topk_overlaps": ([vp, vp, vp, i64, vp, i32, i32, vp, vp, vp, sz, vp], ctypes.c_int),
        "lor_multi_query_workspace_size": ([i64, vp, i32], sz),
        "lor_multi_query_overlap": ([vp, i64, vp, vp, i32, vp, vp, sz, vp], ctypes.c_int),
        "lor_tune_default": ([vp], None),
        "lor_tune_get": ([vp], ctypes.c_int),
        "lor_tune_set": ([vp], ctypes.c_int),
        "lor_autotune_batch": ([vp, vp, i32, vp, vp, vp, i64, vp, sz, i32, vp, vp, vp], ctypes.c_int),
        "lor_rmq_table_elems": ([i64], i64),
        "lor_rmq_row_stride": ([i64], i64),
        "lor_rmq_build": ([vp, i64, vp, i64, vp], ctypes.c_int),
        "lor_rmq_query": ([vp, vp, i64, vp, vp, i64, vp, vp], ctypes.c_int),
        "lor_rmq_block_table_elems": ([i64], i64),
        "lor_rmq_block_build": ([vp, i64, vp, i64, vp], ctypes.c_int),
        "lor_rmq_block_query": ([vp, vp, vp, i64, vp, vp, i64, vp, vp], ctypes.c_int),
        "lor_rmq_block_argmin": ([vp, vp, vp, i64, vp, vp, i64, vp, vp, vp], ctypes.c_int),
        "lor_radix_sort_workspace_size": ([i64], sz),
        "lor_radix_sort_pairs": ([vp, vp, i64, i32, vp, sz, vp], ctypes.c_int),
        "lor_encode_concat64": ([vp, vp, i32, vp, vp, vp], ctypes.c_int),
        "lor_build_sa64_workspace_size": ([i64, i32], sz),
        "lor_build_sa64": ([vp, i64, i32, vp, vp, sz, vp], ctypes.c_int),
        "lor_lcp64_workspace_size": ([i64], sz),
        "lor_lcp64": ([vp, vp, i64, vp, vp, vp, sz, vp], ctypes.c_int),
        "lor_longest_overlap64_workspace_size": ([i64], sz),
        "lor_longest_overlap64": ([vp, vp, i64, vp, i32, vp, vp, i64, vp, sz, vp], ctypes.c_int),
        "lor_rmq_block_query64": ([vp, vp, vp, i64, vp, vp, i64, vp, vp], ctypes.c_int),
        "lor_device_status": ([vp], ctypes.c_int),
        "lor_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "lor_launch_count": ([], ctypes.c_uint64),
        "lor_last_dc3_trace": ([vp, vp, vp, vp, vp, i32], ctypes.c_int),
        "lor_dc3_route_set": ([i32, i32, i32], ctypes.c_int),
        "lor_dc3_route_get": ([vp, vp, vp], ctypes.c_int),
        "lor_test_set_wait": ([ctypes.c_uint64, i32], ctypes.c_int),
        "lor_profile_enable": ([ctypes.c_int], ctypes.c_int),
        "lor_profile_reset": ([], ctypes.c_int),
        "lor_profile_kinds": ([], ctypes.c_int),
        "lor_profile_kind_name": ([ctypes.c_int], ctypes.c_char_p),
        "lor_profile_read": ([ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "lor_server_batch_bytes": ([vp, i32, vp], sz),
        "lor_server_create": ([vp, vp], ctypes.c_int),
        "lor_server_submit": ([vp, vp, i64, vp, i64, ctypes.c_uint64, vp], ctypes.c_int),
        "lor_server_poll": ([vp, vp, i32, i32], ctypes.c_int),
        "lor_server_query": ([vp, i64, vp, vp, i32, vp], ctypes.c_int),
        "lor_server_release": ([vp, i64], ctypes.c_int),
        "lor_server_stats_get": ([vp, vp], ctypes.c_int),
        "lor_server_now": ([vp], ctypes.c_double),
        "lor_server_destroy": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


# ---------------------------------------------------------------- raw C names

def lor_encode_concat(d_ascii, h_lens, nseq, d_text, d_seq_starts, stream):
    return load().lor_encode_concat(d_ascii, h_lens, nseq, d_text, d_seq_starts, stream)


def lor_build_sa_workspace_size(n, sigma):
    return load().lor_build_sa_workspace_size(n, sigma)


def lor_build_sa(d_text, n, sigma, d_sa, d_ws, ws_bytes, stream):
    return load().lor_build_sa(d_text, n, sigma, d_sa, d_ws, ws_bytes, stream)


def lor_build_sa_noalloc(d_text, n, sigma, d_sa, stream):
    return load().lor_build_sa_noalloc(d_text, n, sigma, d_sa, stream)


def lor_lcp_workspace_size(n):
    return load().lor_lcp_workspace_size(n)


def lor_lcp(d_text, d_sa, n, d_isa, d_lcp, d_ws, ws_bytes, stream):
    return load().lor_lcp(d_text, d_sa, n, d_isa, d_lcp, d_ws, ws_bytes, stream)


def lor_longest_overlap_workspace_size(n):
    return load().lor_longest_overlap_workspace_size(n)


def lor_longest_overlap(d_sa, d_lcp, n, d_seq_starts, nseq, d_out, d_pos, pos_cap, d_ws, ws_bytes,
                        stream):
    return load().lor_longest_overlap(d_sa, d_lcp, n, d_seq_starts, nseq, d_out, d_pos, pos_cap,
                                      d_ws, ws_bytes, stream)


def lor_batch_workspace_size(h_lens, npairs):
    return load().lor_batch_workspace_size(h_lens, npairs)


def lor_batch_overlap(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes, stream):
    return load().lor_batch_overlap(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws,
                                    ws_bytes, stream)


def lor_batch_graph_workspace_size(h_lens, npairs):
    return load().lor_batch_graph_workspace_size(h_lens, npairs)


def lor_batch_graph_create(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes, out):
    return load().lor_batch_graph_create(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws,
                                         ws_bytes, out)


def lor_batch_graph_launch(g, stream):
    return load().lor_batch_graph_launch(g, stream)


def lor_batch_graph_kernels(g):
    return load().lor_batch_graph_kernels(g)


def lor_batch_graph_destroy(g):
    return load().lor_batch_graph_destroy(g)


def lor_rmq_table_elems(n):
    return load().lor_rmq_table_elems(n)


def lor_rmq_row_stride(n):
    return load().lor_rmq_row_stride(n)


def table_view(table: torch.Tensor, n: int) -> torch.Tensor:
    """(levels, n) view of a sparse table built for n LCP entries."""
    stride = lor_rmq_row_stride(n)
    return table.view(-1, stride)[:, :n]


def lor_rmq_build(d_lcp, n, d_table, table_elems, stream):
    return load().lor_rmq_build(d_lcp, n, d_table, table_elems, stream)


def lor_rmq_query(d_table, d_isa, n, d_p, d_q, nq, d_out, stream):
    return load().lor_rmq_query(d_table, d_isa, n, d_p, d_q, nq, d_out, stream)


def lor_radix_sort_workspace_size(m):
    return load().lor_radix_sort_workspace_size(m)


def lor_radix_sort_pairs(d_keys, d_vals, m, key_bits, d_ws, ws_bytes, stream):
    return load().lor_radix_sort_pairs(d_keys, d_vals, m, key_bits, d_ws, ws_bytes, stream)


def lor_device_status(stream):
    return load().lor_device_status(stream)


def lor_status_string(status):
    return load().lor_status_string(status).decode()


def lor_launch_count():
    return int(load().lor_launch_count())


# ---------------------------------------------------------------- helpers

def status_string(status: int) -> str:
    try:
        return lor_status_string(status)
    except ImportError:
        return "liblor not loaded"


def _check(rc: int, where: str):
    if rc != LOR_OK:
        raise LorError(rc, where)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor, dtype=None, name="tensor") -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device byte buffer for the *_workspace_size queries (torch's
    allocator returns 512-byte aligned blocks)."""
    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")
    if t.data_ptr() % 256:
        raise RuntimeError("workspace not 256-byte aligned")
    return t


def device_status(stream=None) -> int:
    return lor_device_status(_stream(stream))


def check_device(stream=None, where="device"):
    _check(device_status(stream), where)


def encode_concat(ascii_dev: torch.Tensor, lens, stream=None):
    """ASCII sequences (back to back in one uint8 device tensor) -> text codes
    with terminators, int32 sequence starts and sigma."""
    lens = np.ascontiguousarray(np.asarray(lens, dtype=np.int64))
    nseq = int(lens.size)
    n = int(lens.sum()) + nseq
    dev = ascii_dev.device
    text = torch.empty(n, dtype=torch.uint8, device=dev)
    starts = torch.empty(nseq + 1, dtype=torch.int32, device=dev)
    rc = lor_encode_concat(_ptr(ascii_dev, torch.uint8, "ascii") if ascii_dev.numel() else None,
                           lens.ctypes.data, nseq, _ptr(text), _ptr(starts), _stream(stream))
    _check(rc, "lor_encode_concat")
    return text, starts, nseq + 5


def build_sa(text: torch.Tensor, sigma: int, sa=None, ws=None, stream=None) -> torch.Tensor:
    n = text.numel()
    if sa is None:
        sa = torch.empty(n, dtype=torch.int32, device=text.device)
    need = lor_build_sa_workspace_size(n, sigma)
    if ws is None or ws.numel() < need:
        ws = workspace(need, text.device)
    rc = lor_build_sa(_ptr(text, torch.uint8, "text"), n, sigma, _ptr(sa, torch.int32, "sa"),
                      ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "lor_build_sa")
    return sa


def lcp(text: torch.Tensor, sa: torch.Tensor, isa=None, lcp_out=None, ws=None, stream=None):
    n = text.numel()
    if isa is None:
        isa = torch.empty(n, dtype=torch.int32, device=text.device)
    if lcp_out is None:
        lcp_out = torch.empty(n, dtype=torch.int32, device=text.device)
    need = lor_lcp_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, text.device)
    rc = lor_lcp(_ptr(text, torch.uint8, "text"), _ptr(sa, torch.int32, "sa"), n,
                 _ptr(isa, torch.int32, "isa"), _ptr(lcp_out, torch.int32, "lcp"), ws.data_ptr(),
                 ws.numel(), _stream(stream))
    _check(rc, "lor_lcp")
    return isa, lcp_out


def longest_overlap(sa, lcp_arr, seq_starts, nseq, pos_cap=1 << 16, out=None, pos=None, ws=None,
                    stream=None):
    """Returns (out int32[8] device tensor laid out as lor_overlap, pos device
    tensor of pos_cap entries)."""
    n = sa.numel()
    if out is None:
        out = torch.empty(8, dtype=torch.int32, device=sa.device)
    if pos is None:
        pos = torch.empty(max(int(pos_cap), 1), dtype=torch.int32, device=sa.device)
    need = lor_longest_overlap_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, sa.device)
    rc = lor_longest_overlap(_ptr(sa, torch.int32, "sa"), _ptr(lcp_arr, torch.int32, "lcp"), n,
                             _ptr(seq_starts, torch.int32, "seq_starts"), int(nseq),
                             _ptr(out, torch.int32, "out"), _ptr(pos, torch.int32, "pos"),
                             int(pos_cap), ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "lor_longest_overlap")
    return out, pos


class Batch:
    """Buffers for lor_batch_overlap over a fixed list of pair lengths."""

    def __init__(self, lens, device="cuda", pos_cap=1 << 20):
        self.lens = np.ascontiguousarray(np.asarray(lens, dtype=np.int64))
        if self.lens.size % 2:
            raise ValueError("lens must hold two lengths per pair")
        self.npairs = int(self.lens.size // 2)
        dev = torch.device(device)
        self.out = torch.empty((self.npairs, 8), dtype=torch.int32, device=dev)
        self.pos_off = torch.empty(self.npairs + 1, dtype=torch.int64, device=dev)
        self.pos_cap = int(pos_cap)
        self.pos = torch.empty(max(self.pos_cap, 1), dtype=torch.int32, device=dev)
        need = lor_batch_workspace_size(self.lens.ctypes.data, self.npairs)
        if need == 0:
            raise ValueError("bad pair lengths")
        self.ws = workspace(need, dev)

    def run(self, ascii_dev, stream=None):
        ptr = _ptr(ascii_dev, torch.uint8, "ascii") if ascii_dev.numel() else None
        _check(lor_batch_overlap(ptr, self.lens.ctypes.data, self.npairs, self.out.data_ptr(),
                                 self.pos_off.data_ptr(), self.pos.data_ptr(), self.pos_cap,
                                 self.ws.data_ptr(), self.ws.numel(), _stream(stream)),
               "lor_batch_overlap")
        return self.out, self.pos_off, self.pos

    def results(self):
        """List of per-pair dicts (like overlap_dict) on the host."""
        out = self.out.cpu().numpy()
        off = self.pos_off.cpu().numpy()
        pos = self.pos.cpu().numpy()
        res = []
        for p in range(self.npairs):
            d = dict(zip(OVERLAP_FIELDS, out[p].tolist()))
            a, b = int(off[p]), int(off[p + 1])
            d["positions"] = pos[a:min(b, self.pos_cap)].astype(np.int64)
            res.append(d)
        return res


def topk_overlaps(text, sa, lcp_arr, seq_starts, nseq, K, ws=None, stream=None):
    """lor_topk_overlaps: the K longest left-maximal cross-sequence overlaps as
    a list of dicts (host), largest first."""
    n = text.numel()
    out = torch.empty((K, 8), dtype=torch.int32, device=text.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=text.device)
    need = load().lor_topk_overlaps_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, text.device)
    _check(load().lor_topk_overlaps(_ptr(text, torch.uint8, "text"), _ptr(sa, torch.int32, "sa"),
                                    _ptr(lcp_arr, torch.int32, "lcp"), n, _ptr(seq_starts, torch.int32, "starts"),
                                    int(nseq), int(K), out.data_ptr(), cnt.data_ptr(), ws.data_ptr(), ws.numel(),
                                    _stream(stream)), "lor_topk_overlaps")
    c = int(cnt.item())
    return [dict(zip(OVERLAP_FIELDS, row)) for row in out[:c].cpu().numpy().tolist()]


def multi_query_overlap(ref_dev: torch.Tensor, queries_dev: torch.Tensor, q_lens, out=None, ws=None,
                        stream=None) -> torch.Tensor:
    """lor_multi_query_overlap: per query (length, query_pos, ref_pos, 0) as
    an int32 (nq, 4) device tensor."""
    lens = np.ascontiguousarray(np.asarray(q_lens, dtype=np.int64))
    nq = int(lens.size)
    dev = ref_dev.device if ref_dev.numel() else queries_dev.device
    if out is None:
        out = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    need = load().lor_multi_query_workspace_size(ref_dev.numel(), lens.ctypes.data, nq)
    if need == 0:
        raise ValueError("bad reference or query lengths")
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    rp = _ptr(ref_dev, torch.uint8, "ref") if ref_dev.numel() else None
    qp = _ptr(queries_dev, torch.uint8, "queries") if queries_dev.numel() else None
    _check(load().lor_multi_query_overlap(rp, ref_dev.numel(), qp, lens.ctypes.data, nq, out.data_ptr(),
                                          ws.data_ptr(), ws.numel(), _stream(stream)), "lor_multi_query_overlap")
    return out


class Tune(ctypes.Structure):
    """lor_tune: launch parameters (every value gives the same results)."""
    _fields_ = [("digit_bits", ctypes.c_int32), ("level0_key_bits", ctypes.c_int32),
                ("sort_items_64", ctypes.c_int32), ("sort_items_32", ctypes.c_int32),
                ("merge_items", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def tune_default() -> dict:
    t = Tune()
    load().lor_tune_default(ctypes.byref(t))
    return t.as_dict()


def tune_get() -> dict:
    t = Tune()
    _check(load().lor_tune_get(ctypes.byref(t)), "lor_tune_get")
    return t.as_dict()


def tune_set(**values) -> dict:
    """Set some launch parameters (the others keep their current values)."""
    t = Tune(**{**tune_get(), **values})
    _check(load().lor_tune_set(ctypes.byref(t)), "lor_tune_set")
    return t.as_dict()


_STRATEGIES = {"auto": 0, "sort": 1}
_DOUBLING = {"never": 0, "auto": 1, "force": 2}


def dc3_route_get() -> dict:
    k0, st, db = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().lor_dc3_route_get(ctypes.byref(k0), ctypes.byref(st), ctypes.byref(db)), "lor_dc3_route_get")
    inv_s = {v: k for k, v in _STRATEGIES.items()}
    inv_d = {v: k for k, v in _DOUBLING.items()}
    return {"level0_symbols": int(k0.value), "strategy": inv_s[st.value], "doubling": inv_d[db.value]}


def dc3_route_set(level0_symbols: int = 0, strategy: str = "auto", doubling: str = "auto") -> dict:
    """lor_dc3_route_set: how the suffix array orders its samples (never what
    it returns).  strategy "auto" | "sort"; doubling "never" | "auto" | "force"."""
    _check(load().lor_dc3_route_set(int(level0_symbols), _STRATEGIES[strategy], _DOUBLING[doubling]),
           "lor_dc3_route_set")
    return dc3_route_get()


class dc3_route:
    """Context manager: a DC3 route for the body, the defaults afterwards."""

    def __init__(self, **route):
        self.route = route

    def __enter__(self):
        return dc3_route_set(**self.route)

    def __exit__(self, *exc):
        dc3_route_set()
        return False


def test_set_wait(limit_ns: int = 0, starve_first_tile: bool = False) -> None:
    """lor_test_set_wait: the bounded waits' limit (0 = default 2 s) and the
    switch that withholds the first radix tile's look-back descriptor."""
    _check(load().lor_test_set_wait(int(limit_ns), 1 if starve_first_tile else 0), "lor_test_set_wait")


def autotune_batch(batch: "Batch", ascii_dev, reps: int = 2, stream=None):
    """lor_autotune_batch on a Batch's pairs and buffers; returns (the
    configuration now set, its ms per batch)."""
    best = Tune()
    ms = ctypes.c_double()
    ptr = _ptr(ascii_dev, torch.uint8, "ascii") if ascii_dev.numel() else None
    _check(load().lor_autotune_batch(ptr, batch.lens.ctypes.data, batch.npairs, batch.out.data_ptr(),
                                     batch.pos_off.data_ptr(), batch.pos.data_ptr(), batch.pos_cap,
                                     batch.ws.data_ptr(), batch.ws.numel(), int(reps), _stream(stream),
                                     ctypes.byref(best), ctypes.byref(ms)), "lor_autotune_batch")
    return best.as_dict(), float(ms.value)


class BatchGraph(Batch):
    """lor_batch_graph over a fixed list of pair lengths and a fixed device
    input buffer: the grouped pipeline is captured once into a CUDA graph;
    run() replays it on whatever bases the input buffer holds."""

    def __init__(self, lens, ascii_dev, device="cuda", pos_cap=1 << 20):
        self.lens = np.ascontiguousarray(np.asarray(lens, dtype=np.int64))
        if self.lens.size % 2:
            raise ValueError("lens must hold two lengths per pair")
        self.npairs = int(self.lens.size // 2)
        dev = torch.device(device)
        self.ascii = ascii_dev
        self.out = torch.empty((self.npairs, 8), dtype=torch.int32, device=dev)
        self.pos_off = torch.empty(self.npairs + 1, dtype=torch.int64, device=dev)
        self.pos_cap = int(pos_cap)
        self.pos = torch.empty(max(self.pos_cap, 1), dtype=torch.int32, device=dev)
        need = lor_batch_graph_workspace_size(self.lens.ctypes.data, self.npairs)
        if need == 0:
            raise ValueError("bad pair lengths")
        self.ws = workspace(need, dev)
        ptr = _ptr(ascii_dev, torch.uint8, "ascii") if ascii_dev.numel() else None
        h = ctypes.c_void_p()
        _check(lor_batch_graph_create(ptr, self.lens.ctypes.data, self.npairs, self.out.data_ptr(),
                                      self.pos_off.data_ptr(), self.pos.data_ptr(), self.pos_cap,
                                      self.ws.data_ptr(), self.ws.numel(), ctypes.byref(h)),
               "lor_batch_graph_create")
        self._g = h

    @property
    def kernels(self) -> int:
        return int(lor_batch_graph_kernels(self._g))

    def run(self, ascii_dev=None, stream=None):
        if ascii_dev is not None and ascii_dev.data_ptr() != self.ascii.data_ptr():
            raise ValueError("a batch graph reads the input buffer it was created with")
        _check(lor_batch_graph_launch(self._g, _stream(stream)), "lor_batch_graph_launch")
        return self.out, self.pos_off, self.pos

    def close(self):
        if getattr(self, "_g", None):
            lor_batch_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("workers", ctypes.c_int32),
                ("max_batch_pairs", ctypes.c_int32), ("max_batch_symbols", ctypes.c_int64)]


class Overlap(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in OVERLAP_FIELDS]


class Served(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("batch_pairs", ctypes.c_int32), ("ov", Overlap),
                ("positions", ctypes.POINTER(ctypes.c_int32)), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "released", "batches", "pairs",
                                              "bases", "admission_waits", "queries")] + \
               [(f, ctypes.c_size_t) for f in ("reserved_bytes", "in_use_bytes", "peak_bytes")] + \
               [("pending", ctypes.c_int32), ("in_flight", ctypes.c_int32)]


def server_batch_bytes(lens):
    """(workspace bytes, resident bytes) one batch of these pair lengths takes."""
    lens = np.ascontiguousarray(np.asarray(lens, dtype=np.int64))
    res = ctypes.c_size_t(0)
    work = load().lor_server_batch_bytes(lens.ctypes.data, int(lens.size // 2), ctypes.byref(res))
    return int(work), int(res.value)


class Server:
    """Request server of liblor (lor_server_*): submit pairs, poll results,
    ask LCP queries on a polled request, release it."""

    def __init__(self, budget_bytes, workers=2, max_batch_pairs=512, max_batch_symbols=1 << 28):
        L = load()
        cfg = ServerConfig(int(budget_bytes), int(workers), int(max_batch_pairs), int(max_batch_symbols))
        h = ctypes.c_void_p()
        _check(L.lor_server_create(ctypes.byref(cfg), ctypes.byref(h)), "lor_server_create")
        self._L, self._h = L, h
        self._keep = {}
        self._buf = (Served * 256)()

    def submit_ptr(self, ptr_a, len_a, ptr_b, len_b, tag=0) -> int:
        """Queue a pair given host pointers that stay valid until polled."""
        rid = ctypes.c_int64(0)
        _check(self._L.lor_server_submit(self._h, ptr_a or None, int(len_a), ptr_b or None, int(len_b),
                                         int(tag), ctypes.byref(rid)), "lor_server_submit")
        return int(rid.value)

    def submit(self, a, b, tag=0) -> int:
        """Queue a pair of host uint8 arrays (kept alive until polled)."""
        a = np.ascontiguousarray(a, dtype=np.uint8)
        b = np.ascontiguousarray(b, dtype=np.uint8)
        rid = self.submit_ptr(a.ctypes.data if a.size else None, a.size,
                              b.ctypes.data if b.size else None, b.size, tag)
        self._keep[rid] = (a, b)
        return rid

    def poll(self, timeout_ms=10, cap=256) -> list:
        k = self._L.lor_server_poll(self._h, self._buf, min(cap, len(self._buf)), int(timeout_ms))
        if k < 0:
            raise LorError(k, "lor_server_poll")
        out = []
        for i in range(k):
            r = self._buf[i]
            d = {f: getattr(r.ov, f) for f in OVERLAP_FIELDS}
            n = d["n_pos"] if r.status == LOR_OK else 0
            d["positions"] = (np.ctypeslib.as_array(r.positions, shape=(n,)).astype(np.int64)
                              if n else np.zeros(0, np.int64))
            d.update(id=r.id, tag=r.tag, status=r.status, batch_pairs=r.batch_pairs,
                     t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done)
            self._keep.pop(r.id, None)
            out.append(d)
        return out

    def query(self, rid, p, q) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.int32)
        q = np.ascontiguousarray(q, dtype=np.int32)
        if p.shape != q.shape:
            raise ValueError("p and q differ in length")
        out = np.empty(p.size, dtype=np.int32)
        _check(self._L.lor_server_query(self._h, int(rid), p.ctypes.data, q.ctypes.data, p.size,
                                        out.ctypes.data), "lor_server_query")
        return out

    def release(self, rid):
        _check(self._L.lor_server_release(self._h, int(rid)), "lor_server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._L.lor_server_stats_get(self._h, ctypes.byref(st)), "lor_server_stats_get")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def now(self) -> float:
        return float(self._L.lor_server_now(self._h))

    def close(self):
        if self._h:
            self._L.lor_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def overlap_dict(out: torch.Tensor, pos: torch.Tensor, seq_starts=None) -> dict:
    """Host view of a lor_overlap result (global positions, like the oracle)."""
    vals = out.cpu().tolist()
    d = dict(zip(OVERLAP_FIELDS, vals))
    k = min(d["n_pos"], pos.numel())
    d["positions"] = pos[:k].cpu().numpy().astype(np.int64)
    return d


def rmq_build(lcp_arr: torch.Tensor, table=None, stream=None) -> torch.Tensor:
    n = lcp_arr.numel()
    elems = lor_rmq_table_elems(n)
    if table is None:
        table = torch.empty(elems, dtype=torch.int32, device=lcp_arr.device)
    rc = lor_rmq_build(_ptr(lcp_arr, torch.int32, "lcp"), n, _ptr(table, torch.int32, "table"),
                       table.numel(), _stream(stream))
    _check(rc, "lor_rmq_build")
    return table


def rmq_block_build(lcp_arr: torch.Tensor, table=None, stream=None) -> torch.Tensor:
    """Block-sparse (linear-space) table over an LCP array (lor_rmq_block_build)."""
    n = lcp_arr.numel()
    elems = int(load().lor_rmq_block_table_elems(n))
    if table is None:
        table = torch.empty(elems, dtype=torch.int32, device=lcp_arr.device)
    _check(load().lor_rmq_block_build(_ptr(lcp_arr, torch.int32, "lcp"), n, _ptr(table, torch.int32, "table"),
                                      table.numel(), _stream(stream)), "lor_rmq_block_build")
    return table


def rmq_block_query(table, lcp_arr, isa, p, q, out=None, stream=None) -> torch.Tensor:
    """LCP of suffix pairs through the block-sparse table (lor_rmq_block_query)."""
    if out is None:
        out = torch.empty_like(p)
    _check(load().lor_rmq_block_query(_ptr(table, torch.int32, "table"), _ptr(lcp_arr, torch.int32, "lcp"),
                                      _ptr(isa, torch.int32, "isa"), isa.numel(), _ptr(p, torch.int32, "p"),
                                      _ptr(q, torch.int32, "q"), p.numel(), _ptr(out, torch.int32, "out"),
                                      _stream(stream)), "lor_rmq_block_query")
    return out


def rmq_block_argmin(table, lcp_arr, isa, p, q, stream=None):
    """(value, leftmost rank of the minimum) per suffix pair (lor_rmq_block_argmin)."""
    val = torch.empty_like(p)
    arg = torch.empty_like(p)
    _check(load().lor_rmq_block_argmin(_ptr(table, torch.int32, "table"), _ptr(lcp_arr, torch.int32, "lcp"),
                                       _ptr(isa, torch.int32, "isa"), isa.numel(), _ptr(p, torch.int32, "p"),
                                       _ptr(q, torch.int32, "q"), p.numel(), _ptr(val, torch.int32, "val"),
                                       _ptr(arg, torch.int32, "arg"), _stream(stream)), "lor_rmq_block_argmin")
    return val, arg


def rmq_query(table, isa, p, q, out=None, stream=None) -> torch.Tensor:
    n = isa.numel()
    nq = p.numel()
    if out is None:
        out = torch.empty(nq, dtype=torch.int32, device=isa.device)
    rc = lor_rmq_query(_ptr(table, torch.int32, "table"), _ptr(isa, torch.int32, "isa"), n,
                       _ptr(p, torch.int32, "p"), _ptr(q, torch.int32, "q"), nq,
                       _ptr(out, torch.int32, "out"), _stream(stream))
    _check(rc, "lor_rmq_query")
    return out


# ------------------------------------------------- 64-bit indices (*64 calls)

def encode_concat64(ascii_dev: torch.Tensor, lens, stream=None):
    """As encode_concat, with int64 sequence starts (lor_encode_concat64)."""
    lens = np.ascontiguousarray(np.asarray(lens, dtype=np.int64))
    nseq = int(lens.size)
    n = int(lens.sum()) + nseq
    dev = ascii_dev.device
    text = torch.empty(n, dtype=torch.uint8, device=dev)
    starts = torch.empty(nseq + 1, dtype=torch.int64, device=dev)
    rc = load().lor_encode_concat64(_ptr(ascii_dev, torch.uint8, "ascii") if ascii_dev.numel() else None,
                                    lens.ctypes.data, nseq, _ptr(text), _ptr(starts), _stream(stream))
    _check(rc, "lor_encode_concat64")
    return text, starts, nseq + 5


def build_sa64(text: torch.Tensor, sigma: int, sa=None, ws=None, stream=None) -> torch.Tensor:
    """int64 suffix array (lor_build_sa64)."""
    n = text.numel()
    if sa is None:
        sa = torch.empty(n, dtype=torch.int64, device=text.device)
    need = load().lor_build_sa64_workspace_size(n, sigma)
    if need == 0:
        raise LorError(LOR_ERR_TOO_LARGE if n > LOR_MAX_N64 else LOR_ERR_INVALID_ARG, "lor_build_sa64")
    if ws is None or ws.numel() < need:
        ws = workspace(need, text.device)
    rc = load().lor_build_sa64(_ptr(text, torch.uint8, "text"), n, sigma, _ptr(sa, torch.int64, "sa"),
                               ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "lor_build_sa64")
    return sa


def lcp64(text: torch.Tensor, sa: torch.Tensor, isa=None, lcp_out=None, ws=None, stream=None):
    """(int64 ISA, int32 LCP) from an int64 suffix array (lor_lcp64)."""
    n = text.numel()
    if isa is None:
        isa = torch.empty(n, dtype=torch.int64, device=text.device)
    if lcp_out is None:
        lcp_out = torch.empty(n, dtype=torch.int32, device=text.device)
    need = load().lor_lcp64_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, text.device)
    rc = load().lor_lcp64(_ptr(text, torch.uint8, "text"), _ptr(sa, torch.int64, "sa"), n,
                          _ptr(isa, torch.int64, "isa"), _ptr(lcp_out, torch.int32, "lcp"), ws.data_ptr(),
                          ws.numel(), _stream(stream))
    _check(rc, "lor_lcp64")
    return isa, lcp_out


OVERLAP64_FIELDS = ("length", "seq_a", "seq_b", "reserved", "rank", "pos_a", "pos_b", "n_pos")


def longest_overlap64(sa, lcp_arr, seq_starts, nseq, pos_cap=1 << 16, out=None, pos=None, ws=None, stream=None):
    """(out: 48-byte lor_overlap64 as a uint8 device tensor, pos: int64 device
    tensor of pos_cap entries) (lor_longest_overlap64)."""
    n = sa.numel()
    if out is None:
        out = torch.empty(48, dtype=torch.uint8, device=sa.device)
    if pos is None:
        pos = torch.empty(max(int(pos_cap), 1), dtype=torch.int64, device=sa.device)
    need = load().lor_longest_overlap64_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, sa.device)
    rc = load().lor_longest_overlap64(_ptr(sa, torch.int64, "sa"), _ptr(lcp_arr, torch.int32, "lcp"), n,
                                      _ptr(seq_starts, torch.int64, "seq_starts"), int(nseq), _ptr(out),
                                      _ptr(pos, torch.int64, "pos"), int(pos_cap), ws.data_ptr(), ws.numel(),
                                      _stream(stream))
    _check(rc, "lor_longest_overlap64")
    return out, pos


def overlap64_dict(out: torch.Tensor, pos: torch.Tensor) -> dict:
    """Host view of a lor_overlap64 result, keyed like overlap_dict."""
    raw = out.cpu().numpy().tobytes()
    head = np.frombuffer(raw[:16], dtype=np.int32).tolist()
    tail = np.frombuffer(raw[16:48], dtype=np.int64).tolist()
    d = dict(zip(OVERLAP64_FIELDS, head + tail))
    k = min(d["n_pos"], pos.numel())
    d["positions"] = pos[:k].cpu().numpy().astype(np.int64)
    return d


def rmq_block_query64(table, lcp_arr, isa, p, q, out=None, stream=None) -> torch.Tensor:
    """LCP of suffix pairs of a 64-bit text through its block table
    (lor_rmq_block_query64): int64 ISA, positions and answers."""
    if out is None:
        out = torch.empty(p.numel(), dtype=torch.int64, device=p.device)
    _check(load().lor_rmq_block_query64(_ptr(table, torch.int32, "table"), _ptr(lcp_arr, torch.int32, "lcp"),
                                        _ptr(isa, torch.int64, "isa"), isa.numel(), _ptr(p, torch.int64, "p"),
                                        _ptr(q, torch.int64, "q"), p.numel(), _ptr(out, torch.int64, "out"),
                                        _stream(stream)), "lor_rmq_block_query64")
    return out


def radix_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int, stream=None):
    """Stable in-place sort of (int64-stored uint64 keys, int32-stored uint32
    values) by the low key_bits bits."""
    m = keys.numel()
    ws = workspace(lor_radix_sort_workspace_size(m), keys.device)
    rc = lor_radix_sort_pairs(_ptr(keys, torch.int64, "keys"), _ptr(vals, torch.int32, "vals"), m,
                              int(key_bits), ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "lor_radix_sort_pairs")
    return keys, vals


def last_dc3_trace():
    cap = 128
    n = np.zeros(cap, np.int64)
    names = np.zeros(cap, np.int64)
    bits = np.zeros(cap, np.int32)
    strat = np.zeros(cap, np.int32)
    dups = np.zeros(cap, np.int64)
    cnt = load().lor_last_dc3_trace(n.ctypes.data, names.ctypes.data, bits.ctypes.data,
                                    strat.ctypes.data, dups.ctypes.data, cap)
    cnt = min(cnt, cap)
    kinds = ("sort", "dense", "parent", "doubling")
    return [dict(n=int(n[i]), names=int(names[i]), key_bits=int(bits[i]),
                 strategy=kinds[int(strat[i])], dups=int(dups[i])) for i in range(cnt)]


def profile_enable(on=True):
    _check(load().lor_profile_enable(1 if on else 0), "lor_profile_enable")


def profile_reset():
    _check(load().lor_profile_reset(), "lor_profile_reset")


def profile_read() -> dict:
    L = load()
    out = {}
    for k in range(L.lor_profile_kinds()):
        c = ctypes.c_int64()
        ms = ctypes.c_double()
        b = ctypes.c_double()
        _check(L.lor_profile_read(k, ctypes.byref(c), ctypes.byref(ms), ctypes.byref(b)),
               "lor_profile_read")
        if c.value:
            out[L.lor_profile_kind_name(k).decode()] = dict(launches=c.value, ms=ms.value,
                                                            bytes=b.value)
    return out


class Pipeline:
    """Device-resident buffers for repeated runs of the whole path on texts of
    one length: encode -> SA -> ISA/LCP -> overlap -> sparse table -> queries."""

    def __init__(self, lens, device="cuda", pos_cap=1 << 16, with_rmq=True):
        self.lens = np.asarray(lens, dtype=np.int64)
        self.nseq = int(self.lens.size)
        self.n = int(self.lens.sum()) + self.nseq
        self.sigma = self.nseq + 5
        dev = torch.device(device)
        n = self.n
        self.text = torch.empty(n, dtype=torch.uint8, device=dev)
        self.starts = torch.empty(self.nseq + 1, dtype=torch.int32, device=dev)
        self.sa = torch.empty(n, dtype=torch.int32, device=dev)
        self.isa = torch.empty(n, dtype=torch.int32, device=dev)
        self.lcp = torch.empty(n, dtype=torch.int32, device=dev)
        self.out = torch.empty(8, dtype=torch.int32, device=dev)
        self.pos_cap = int(pos_cap)
        self.pos = torch.empty(max(self.pos_cap, 1), dtype=torch.int32, device=dev)
        ws_bytes = max(lor_build_sa_workspace_size(n, self.sigma),
                       lor_longest_overlap_workspace_size(n), lor_lcp_workspace_size(n))
        self.ws = workspace(ws_bytes, dev)
        self.table = (torch.empty(lor_rmq_table_elems(n), dtype=torch.int32, device=dev)
                      if with_rmq else None)

    def run(self, ascii_dev, p=None, q=None, answers=None, stream=None):
        s = _stream(stream)
        _check(lor_encode_concat(_ptr(ascii_dev, torch.uint8, "ascii"), self.lens.ctypes.data,
                                 self.nseq, self.text.data_ptr(), self.starts.data_ptr(), s),
               "lor_encode_concat")
        _check(lor_build_sa(self.text.data_ptr(), self.n, self.sigma, self.sa.data_ptr(),
                            self.ws.data_ptr(), self.ws.numel(), s), "lor_build_sa")
        _check(lor_lcp(self.text.data_ptr(), self.sa.data_ptr(), self.n, self.isa.data_ptr(),
                       self.lcp.data_ptr(), self.ws.data_ptr(), self.ws.numel(), s), "lor_lcp")
        _check(lor_longest_overlap(self.sa.data_ptr(), self.lcp.data_ptr(), self.n,
                                   self.starts.data_ptr(), self.nseq, self.out.data_ptr(),
                                   self.pos.data_ptr(), self.pos_cap, self.ws.data_ptr(),
                                   self.ws.numel(), s), "lor_longest_overlap")
        if self.table is not None:
            _check(lor_rmq_build(self.lcp.data_ptr(), self.n, self.table.data_ptr(),
                                 self.table.numel(), s), "lor_rmq_build")
            if p is not None:
                _check(lor_rmq_query(self.table.data_ptr(), self.isa.data_ptr(), self.n,
                                     _ptr(p, torch.int32, "p"), _ptr(q, torch.int32, "q"),
                                     p.numel(), _ptr(answers, torch.int32, "answers"), s),
                       "lor_rmq_query")
        return self.out, self.pos
