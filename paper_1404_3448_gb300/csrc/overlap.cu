// overlap.cu -- longest overlap region from SA + LCP (Section 3: the longest
// common prefix of suffixes of two sequences and its positions in the suffix
// array).
//
//   1. argmax: L = max LCP[k] over rank-adjacent suffixes from different
//      sequences, smallest such k; a warp-shuffle max of the packed key
//      (LCP << 32 | ~k), a block max and one 64-bit atomicMax per block.
//   2. positions: rank runs with adjacent LCP >= L (run ids by a look-back
//      scan), a run qualifies when it holds a cross-sequence adjacent pair,
//      every member of a qualifying run is compacted out, and the list is
//      radix sorted ascending.
#include "radix.cuh"

LOR_DEFINE_TU_STATUS(lor_status_overlap)

namespace lor {
namespace {

constexpr int kOvThreads = 256;
constexpr int kOvItems = 8;
constexpr int kOvTile = kOvThreads * kOvItems;

struct OvLayout {
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t run_id = 0, qual = 0, ka = 0, kb = 0, va = 0, vb = 0, total = 0;
};

OvLayout ov_layout(int64_t n) {
    OvLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(n);
    L.lookback = take(L.lookback_bytes);
    L.run_id = take(sizeof(int32_t) * size_t(n));
    L.qual = take(size_t(n));
    L.ka = take(sizeof(uint32_t) * size_t(n));
    L.kb = take(sizeof(uint32_t) * size_t(n));
    L.va = take(sizeof(uint32_t) * size_t(n));
    L.vb = take(sizeof(uint32_t) * size_t(n));
    L.total = off;
    return L;
}

// Sequence holding text position p: largest s with starts[s] <= p.
__device__ __forceinline__ int seq_of(const int32_t *starts, int nseq, int32_t p) {
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_ov_argmax(const int32_t *__restrict__ sa,
                                                   const int32_t *__restrict__ lcp, int64_t n,
                                                   const int32_t *__restrict__ starts, int nseq,
                                                   unsigned long long *best) {
    __shared__ int32_t sst[LOR_MAX_SEQ + 1];
    __shared__ unsigned long long wbest[8];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    unsigned long long my = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = 1 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
        const int32_t a = sa[k - 1], b = sa[k];
        if (seq_of(sst, nseq, a) != seq_of(sst, nseq, b)) {
            const unsigned long long key =
                (static_cast<unsigned long long>(uint32_t(lcp[k])) << 32) | (0xFFFFFFFFull - uint64_t(k));
            my = key > my ? key : my;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, my, d);
        my = o > my ? o : my;
    }
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = my;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) b = wbest[w] > b ? wbest[w] : b;
        if (b) atomicMax(best, b);
    }
}

__device__ __forceinline__ int32_t best_len(const unsigned long long *best) {
    return int32_t(*best >> 32);
}

// run_id[k] = number of run starts in [0, k] minus one; a run starts at k = 0
// and wherever LCP[k] < L.
__global__ void __launch_bounds__(kOvThreads) k_ov_runs(const int32_t *__restrict__ lcp, int64_t n,
                                                        const unsigned long long *best,
                                                        int32_t *__restrict__ run_id, uint64_t *lb,
                                                        unsigned long long *ctr,
                                                        unsigned long long tile_base, uint32_t epoch,
                                                        int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kOvThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int32_t L = best_len(best);
    if (L <= 0) return;
    const int64_t tile = s_tile;
    const int64_t base = tile * kOvTile + int64_t(tid) * kOvItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kOvItems; ++i) {
        const int64_t k = base + i;
        if (k < n) {
            const uint32_t f = (k == 0 || lcp[k] < L) ? 1u : 0u;
            flags |= f << i;
            cnt += f;
        }
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kOvThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) s_prefix = p;
    }
    __syncthreads();
    uint32_t id = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kOvItems; ++i) {
        const int64_t k = base + i;
        if (k < n) {
            id += (flags >> i) & 1u;
            run_id[k] = int32_t(id) - 1;
        }
    }
}

// A run qualifies when it holds an adjacent pair from different sequences.
__global__ void k_ov_qual(const int32_t *__restrict__ sa, const int32_t *__restrict__ lcp, int64_t n,
                          const int32_t *__restrict__ starts, int nseq,
                          const unsigned long long *best, const int32_t *__restrict__ run_id,
                          uint8_t *__restrict__ qual) {
    __shared__ int32_t sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    const int32_t L = best_len(best);
    if (L <= 0) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = 1 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
        if (lcp[k] >= L && seq_of(sst, nseq, sa[k - 1]) != seq_of(sst, nseq, sa[k]))
            qual[run_id[k]] = 1;
    }
}

// Members of qualifying runs, compacted in rank order.
__global__ void __launch_bounds__(kOvThreads) k_ov_members(
    const int32_t *__restrict__ sa, int64_t n, const unsigned long long *best,
    const int32_t *__restrict__ run_id, const uint8_t *__restrict__ qual, uint32_t *__restrict__ out,
    uint32_t *count, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base,
    int64_t ntiles, uint32_t epoch, int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kOvThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int32_t L = best_len(best);
    if (L <= 0) return;
    const int64_t tile = s_tile;
    const int64_t base = tile * kOvTile + int64_t(tid) * kOvItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kOvItems; ++i) {
        const int64_t k = base + i;
        if (k < n && qual[run_id[k]]) {
            flags |= 1u << i;
            cnt++;
        }
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kOvThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) {
            s_prefix = p;
            if (tile == ntiles - 1) *count = p + agg;
        }
    }
    __syncthreads();
    uint32_t o = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kOvItems; ++i) {
        if ((flags >> i) & 1u) out[o++] = uint32_t(sa[base + i]);
    }
}

__global__ void k_ov_result(const int32_t *__restrict__ sa, const int32_t *__restrict__ starts, int nseq,
                            const unsigned long long *best, const uint32_t *count, lor_overlap *out) {
    __shared__ int32_t sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    lor_overlap r;
    const unsigned long long b = *best;
    const int32_t L = int32_t(b >> 32);
    r.reserved = 0;
    if (L <= 0) {
        r.length = 0;
        r.rank = r.seq_a = r.pos_a = r.seq_b = r.pos_b = -1;
        r.n_pos = 0;
    } else {
        const int64_t k = int64_t(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
        int32_t a = sa[k - 1], c = sa[k];
        int sa_ = seq_of(sst, nseq, a), sc_ = seq_of(sst, nseq, c);
        if (sa_ > sc_) {
            const int32_t t = a; a = c; c = t;
            const int u = sa_; sa_ = sc_; sc_ = u;
        }
        r.length = L;
        r.rank = int32_t(k);
        r.seq_a = sa_;
        r.pos_a = a - sst[sa_];
        r.seq_b = sc_;
        r.pos_b = c - sst[sc_];
        r.n_pos = int32_t(*count);
    }
    *out = r;
}

__global__ void k_copy_u32_i32(const uint32_t *__restrict__ src, int32_t *__restrict__ dst, int64_t m) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) dst[i] = int32_t(src[i]);
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_longest_overlap_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return ov_layout(n).total;
}

extern "C" int lor_longest_overlap(const int32_t *d_sa, const int32_t *d_lcp, int64_t n,
                                   const int32_t *d_seq_starts, int32_t nseq, lor_overlap *d_out,
                                   int32_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                                   lor_stream_t stream) {
    if (!d_sa || !d_lcp || !d_seq_starts || !d_out || n < 1 || pos_cap < 0) return LOR_ERR_INVALID_ARG;
    if (nseq < 1 || nseq > LOR_MAX_SEQ) return LOR_ERR_INVALID_ARG;
    if (pos_cap > 0 && !d_pos) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const OvLayout L = ov_layout(n);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    char *ws = (char *)d_ws;
    unsigned long long *best = (unsigned long long *)(ws + L.ctrl);
    uint32_t *count = (uint32_t *)(ws + L.ctrl + 8);
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl + 64);
    rs.max_tiles = cdiv(n, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    int32_t *run_id = (int32_t *)(ws + L.run_id);
    uint8_t *qual = (uint8_t *)(ws + L.qual);
    uint32_t *ka = (uint32_t *)(ws + L.ka), *kb = (uint32_t *)(ws + L.kb);
    uint32_t *va = (uint32_t *)(ws + L.va), *vb = (uint32_t *)(ws + L.vb);

    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    LOR_CUDA_TRY(cudaMemsetAsync(qual, 0, size_t(n), s));
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 8, s);
        const unsigned grid = unsigned(min64(cdiv(n, 256), 152 * 16));
        k_ov_argmax<<<grid, 256, 0, s>>>(d_sa, d_lcp, n, d_seq_starts, nseq, best);
    }
    LOR_LAUNCH_CHECK();
    const int64_t ntiles = cdiv(n, kOvTile);
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 8, s);
        rs.epoch++;
        k_ov_runs<<<unsigned(ntiles), kOvThreads, 0, s>>>(d_lcp, n, best, run_id, rs.lookback,
                                                         rs.tile_ctr, rs.tile_base, rs.epoch, status);
    }
    LOR_LAUNCH_CHECK();
    rs.tile_base += (unsigned long long)ntiles;
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 12, s);
        const unsigned grid = unsigned(min64(cdiv(n, 256), 152 * 16));
        k_ov_qual<<<grid, 256, 0, s>>>(d_sa, d_lcp, n, d_seq_starts, nseq, best, run_id, qual);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 5, s);
        rs.epoch++;
        k_ov_members<<<unsigned(ntiles), kOvThreads, 0, s>>>(d_sa, n, best, run_id, qual, ka, count,
                                                            rs.lookback, rs.tile_ctr, rs.tile_base,
                                                            ntiles, rs.epoch, status);
    }
    LOR_LAUNCH_CHECK();
    rs.tile_base += (unsigned long long)ntiles;
    uint32_t h_count = 0;
    LOR_CUDA_TRY(cudaMemcpyAsync(&h_count, count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t m = int64_t(h_count);
    uint32_t *kr = ka, *vr = va;
    if (m > 1) {
        const int bits = bit_width_u64(uint64_t(n - 1));
        const int rc = radix_sort_pairs<uint32_t>(rs, ka, va, kb, vb, m, 0, bits, true, &kr, &vr);
        if (rc) return rc;
    }
    k_ov_result<<<1, 256, 0, s>>>(d_sa, d_seq_starts, nseq, best, count, d_out);
    LOR_LAUNCH_CHECK();
    const int64_t ncopy = m < pos_cap ? m : pos_cap;
    if (ncopy > 0) {
        k_copy_u32_i32<<<unsigned(cdiv(ncopy, 256)), 256, 0, s>>>(kr, d_pos, ncopy);
        LOR_LAUNCH_CHECK();
    }
    return LOR_OK;
}
