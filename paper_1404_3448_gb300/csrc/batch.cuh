// batch.cuh -- the grouped pipeline (one suffix array over the texts of up to
// 125 sequence pairs, split into per-pair blocks) as used by the batched entry
// point and by the request server.
#pragma once

#include "common.cuh"

namespace lor {

// Pairs per group and their sequences.  Every pair's text inside a group is
// its own S1#S2$ (the terminator codes are shared by all pairs of the group),
// so the group size is not bound by the number of terminator codes.
constexpr int kPairsPerGroup = 512;
constexpr int kGroupSeqs = 2 * kPairsPerGroup;
constexpr int64_t kGroupSymbolCap = int64_t(1) << 28;

// Offsets (bytes from the workspace start) of one group's buffers.  The text,
// terminator starts and suffix array come first; everything after `region` is
// the suffix-array workspace while DC3 runs and the post-SA buffers after it.
struct BatchLayout {
    size_t text = 0, starts = 0, sa = 0, region = 0, total = 0;
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t pk = 0, pk2 = 0, sa2 = 0, ip = 0, isa = 0, plcp = 0, lcp = 0, run_id = 0, qual = 0;
    size_t mem = 0, kb = 0, va = 0, vb = 0, packed = 0, bstart = 0, best = 0, cnt = 0, post = 0;
};

BatchLayout batch_layout(int64_t nmax);

// lor_build_sa with, when graph_ctr_pool is given, no host round trip at all
// (for stream capture): level 0 and then enqueued doubling rounds, with the
// tile counters of device-sized launches taken from the pool (graph_pool_size
// zeroed counters; the call zeroes them itself first).
int build_sa_impl(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa, void *d_ws, size_t ws_bytes,
                  cudaStream_t stream, unsigned long long *graph_ctr_pool, int graph_pool_size);

// Where one group writes its results: np overlap records, np + 1 position
// offsets (starting at pos_base) and its positions at pos[pos_base ...]
// (positions at or beyond pos_cap are counted but not stored).
struct GroupOutputs {
    lor_overlap *out;
    int64_t *pos_off;
    int32_t *pos;
    int64_t pos_cap;
    int64_t pos_base;
};

// Graph mode of batch_group (work captured into a CUDA graph): the counter
// pools of the suffix array and of the rest, the device-held first position
// slot of the group (advanced by the group's count), and pinned host memory
// for the group's sequence starts that lives as long as the graph.
struct GroupGraph {
    unsigned long long *sa_pool;
    int sa_pool_size;
    unsigned long long *post_pool;
    int post_pool_size;
    int64_t *pos_base;
    int32_t *h_starts;
};

// Runs one group of np pairs (ASCII bases of all 2*np sequences back to back
// at d_ascii, lengths h_lens[0 .. 2*np), text length n = sum + 2*np) on
// stream s.  On return (LOR_OK) the group's results are enqueued, *h_found
// holds its position count, and the workspace still holds the group's text,
// terminator starts, per-pair ISA (ws + L.isa: rank of every text position in
// the blocked suffix array) and LCP (ws + L.lcp, 0 at every block head).
int batch_group(const uint8_t *d_ascii, const int64_t *h_lens, int np, int64_t n, char *ws, size_t ws_bytes,
                const BatchLayout &L, int64_t nmax, const GroupOutputs &o, int64_t *h_found, cudaStream_t s,
                const GroupGraph *g = nullptr);

}  // namespace lor
