// overlap.cu -- longest overlap region from SA + LCP (Section 3: the longest
// common prefix of suffixes of two sequences and its positions in the suffix
// array).
//
//   1. argmax: L = max LCP[k] over rank-adjacent suffixes from different
//      sequences, smallest such k; a warp-shuffle max of the packed key
//      (LCP << 32 | ~k), a block max and one 64-bit atomicMax per block.
//   2. positions: the ranks k with LCP[k] >= L ("hits") are compacted in
//      rank order; consecutive hits k_a .. k_b form one run of ranks
//      k_a - 1 .. k_b (all suffixes sharing the length-L prefix); a run
//      qualifies when one of its adjacent pairs comes from two sequences,
//      every member of a qualifying run is emitted, and the list is radix
//      sorted ascending.  Only the hits (usually a handful) are touched after
//      the compaction.
#include "radix.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_overlap)

namespace lor {
namespace {

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
template <typename StT, typename PT>
__device__ __forceinline__ int seq_of(const StT *starts, int nseq, PT p) {
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Candidate rank k of the argmax: keeps the larger packed key.
template <typename StT, typename SaT>
__device__ __forceinline__ void ov_consider(unsigned long long &my, const StT *sst, int nseq, SaT a, SaT b, int32_t l,
                                           int64_t k) {
    if (uint32_t(l) < uint32_t(my >> 32)) return;  // cannot win: skip the sequence lookups
    if (seq_of(sst, nseq, a) != seq_of(sst, nseq, b)) {
        const unsigned long long key =
            (static_cast<unsigned long long>(uint32_t(l)) << 32) | (0xFFFFFFFFull - uint64_t(k));
        my = key > my ? key : my;
    }
}

// vec: SA and LCP are 16-byte aligned, so four ranks are read per load
// (int32 suffix arrays only).
template <typename SaT, typename StT>
__global__ void __launch_bounds__(256) k_ov_argmax(const SaT *__restrict__ sa,
                                                   const int32_t *__restrict__ lcp, int64_t n,
                                                   const StT *__restrict__ starts, int nseq, int vec,
                                                   unsigned long long *best) {
    __shared__ StT sst[LOR_MAX_SEQ + 1];
    __shared__ unsigned long long wbest[8];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    unsigned long long my = 0;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t k0 = 1;
    if constexpr (sizeof(SaT) == 4) {
        if (vec) {
            const int64_t nv = n / 4;
            for (int64_t v = tid; v < nv; v += stride) {
                const int4 s4 = reinterpret_cast<const int4 *>(sa)[v];
                const int4 l4 = reinterpret_cast<const int4 *>(lcp)[v];
                const int64_t k = 4 * v;
                if (k > 0) ov_consider(my, sst, nseq, sa[k - 1], s4.x, l4.x, k);
                ov_consider(my, sst, nseq, s4.x, s4.y, l4.y, k + 1);
                ov_consider(my, sst, nseq, s4.y, s4.z, l4.z, k + 2);
                ov_consider(my, sst, nseq, s4.z, s4.w, l4.w, k + 3);
            }
            k0 = nv * 4 > 1 ? nv * 4 : 1;
        }
    }
    for (int64_t k = k0 + tid; k < n; k += stride) ov_consider(my, sst, nseq, sa[k - 1], sa[k], lcp[k], k);
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

// Hits: ranks k >= 1 with LCP[k] >= L, appended in any order (a warp
// reserves its slots with one atomic); they are sorted afterwards.
__device__ __forceinline__ void ov_append(bool hit, uint32_t k, uint32_t *hits, uint32_t *count) {
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(int(mask)) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, uint32_t(__popc(mask)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) hits[base + __popc(mask & ((1u << lane) - 1u))] = k;
}

__global__ void __launch_bounds__(256) k_ov_hits(const int32_t *__restrict__ lcp, int64_t n, int vec,
                                                 const unsigned long long *best, uint32_t *__restrict__ hits,
                                                 uint32_t *count) {
    const int32_t L = best_len(best);
    if (L <= 0) return;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t k0 = 0;
    if (vec) {
        const int64_t nv = n / 4;
        const int64_t nvr = (nv + 31) & ~int64_t(31);  // whole warps iterate together
        for (int64_t v = tid; v < nvr; v += stride) {
            int4 l4 = make_int4(0, 0, 0, 0);
            if (v < nv) l4 = reinterpret_cast<const int4 *>(lcp)[v];
            const uint32_t k = uint32_t(4 * v);
            ov_append(v < nv && k > 0 && l4.x >= L, k, hits, count);
            ov_append(v < nv && l4.y >= L, k + 1, hits, count);
            ov_append(v < nv && l4.z >= L, k + 2, hits, count);
            ov_append(v < nv && l4.w >= L, k + 3, hits, count);
        }
        k0 = nv * 4;
    }
    const int64_t rest = n - k0;
    const int64_t restr = (rest + 31) & ~int64_t(31);
    for (int64_t x = tid; x < restr; x += stride) {
        const int64_t k = k0 + x;
        ov_append(x < rest && k > 0 && lcp[k] >= L, uint32_t(k), hits, count);
    }
}

__device__ __forceinline__ bool hit_starts_run(const uint32_t *hits, int64_t i) {
    return i == 0 || hits[i] != hits[i - 1] + 1;
}

// Run ids of the hits; a run qualifies when one of its hits pairs suffixes
// of two sequences.
template <typename SaT, typename StT>
__global__ void __launch_bounds__(kScanThreads) k_ov_hit_runs(
    const SaT *__restrict__ sa, const uint32_t *__restrict__ hits, int64_t c,
    const StT *__restrict__ starts, int nseq, uint32_t *__restrict__ run, uint8_t *__restrict__ qual,
    uint32_t *n_runs, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch,
    int *status) {
    __shared__ StT sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    tile_names(
        c, [&](int64_t i) { return hit_starts_run(hits, i); },
        [&](int64_t i, uint32_t r) {
            run[i] = r - 1;
            const uint32_t k = hits[i];
            if (seq_of(sst, nseq, sa[k - 1]) != seq_of(sst, nseq, sa[k])) qual[r - 1] = 1;
        },
        n_runs, lb, ctr, tile_base, epoch, status);
}

// Members of qualifying runs in rank order: a run's first hit k adds SA[k-1]
// and SA[k], every other hit adds SA[k] (positions < 2^32 as uint32).
template <typename SaT>
__global__ void __launch_bounds__(kScanThreads) k_ov_hit_members(
    const SaT *__restrict__ sa, const uint32_t *__restrict__ hits, int64_t c,
    const uint32_t *__restrict__ run, const uint8_t *__restrict__ qual, uint32_t *__restrict__ out,
    uint32_t *count, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch,
    int *status, int64_t ntiles) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    uint32_t cnt = 0;
    uint32_t two = 0, one = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t x = base + i;
        if (x < c && qual[run[x]]) {
            if (hit_starts_run(hits, x)) {
                two |= 1u << i;
                cnt += 2;
            } else {
                one |= 1u << i;
                cnt += 1;
            }
        }
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
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
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t x = base + i;
        if ((two >> i) & 1u) out[o++] = uint32_t(sa[hits[x] - 1]);
        if (((two | one) >> i) & 1u) out[o++] = uint32_t(sa[hits[x]]);
    }
}

// OutT: lor_overlap (int32 fields) or lor_overlap64 (int64 rank, offsets
// and count).
template <typename SaT, typename StT, typename OutT>
__global__ void k_ov_result(const SaT *__restrict__ sa, const StT *__restrict__ starts, int nseq,
                            const unsigned long long *best, const uint32_t *count, OutT *out) {
    __shared__ StT sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    OutT r;
    const unsigned long long b = *best;
    const int32_t L = int32_t(b >> 32);
    r.reserved = 0;
    if (L <= 0) {
        r.length = 0;
        r.rank = -1;
        r.seq_a = r.seq_b = -1;
        r.pos_a = r.pos_b = -1;
        r.n_pos = 0;
    } else {
        const int64_t k = int64_t(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
        SaT a = sa[k - 1], c = sa[k];
        int sa_ = seq_of(sst, nseq, a), sc_ = seq_of(sst, nseq, c);
        if (sa_ > sc_) {
            const SaT t = a; a = c; c = t;
            const int u = sa_; sa_ = sc_; sc_ = u;
        }
        r.length = L;
        r.rank = decltype(r.rank)(k);
        r.seq_a = sa_;
        r.pos_a = decltype(r.pos_a)(a - sst[sa_]);
        r.seq_b = sc_;
        r.pos_b = decltype(r.pos_b)(c - sst[sc_]);
        r.n_pos = decltype(r.n_pos)(*count);
    }
    *out = r;
}

template <typename PosT>
__global__ void k_copy_u32(const uint32_t *__restrict__ src, PosT *__restrict__ dst, int64_t m) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) dst[i] = PosT(src[i]);
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_longest_overlap_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return ov_layout(n).total;
}

namespace lor {
namespace {

template <typename SaT, typename StT, typename OutT, typename PosT>
int longest_overlap_impl(const SaT *d_sa, const int32_t *d_lcp, int64_t n, const StT *d_seq_starts, int32_t nseq,
                         OutT *d_out, PosT *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                         lor_stream_t stream, int64_t max_n) {
    if (!d_sa || !d_lcp || !d_seq_starts || !d_out || n < 1 || pos_cap < 0) return LOR_ERR_INVALID_ARG;
    if (nseq < 1 || nseq > LOR_MAX_SEQ) return LOR_ERR_INVALID_ARG;
    if (pos_cap > 0 && !d_pos) return LOR_ERR_INVALID_ARG;
    if (n > max_n) return LOR_ERR_TOO_LARGE;
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

    uint32_t *hits = (uint32_t *)run_id, *run = kb;
    uint32_t *n_runs = (uint32_t *)(ws + L.ctrl + 16);
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 8, s);
        const unsigned grid = unsigned(min64(cdiv(n, 1024), 152 * 16));
        const int vec = sizeof(SaT) == 4 && ((uintptr_t(d_sa) | uintptr_t(d_lcp)) & 15) == 0;
        k_ov_argmax<SaT, StT><<<grid, 256, 0, s>>>(d_sa, d_lcp, n, d_seq_starts, nseq, vec, best);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 4, s);
        const int vec = (uintptr_t(d_lcp) & 15) == 0;
        k_ov_hits<<<unsigned(min64(cdiv(n, 1024), 152 * 16)), 256, 0, s>>>(d_lcp, n, vec, best, hits, count);
    }
    LOR_LAUNCH_CHECK();
    uint32_t h_hits = 0;
    LOR_CUDA_TRY(cudaMemcpyAsync(&h_hits, count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t c = int64_t(h_hits);
    uint32_t h_count = 0;
    if (c > 1) {
        uint32_t *hr, *hv;
        const int rc = radix_sort_pairs<uint32_t>(rs, hits, va, kb, vb, c, 0, bit_width_u64(uint64_t(n - 1)), true,
                                                  &hr, &hv);
        if (rc) return rc;
        if (hr != hits)
            LOR_CUDA_TRY(cudaMemcpyAsync(hits, hr, sizeof(uint32_t) * size_t(c), cudaMemcpyDeviceToDevice, s));
    }
    if (c > 0) {
        const int64_t ct = cdiv(c, kScanTile);
        LOR_CUDA_TRY(cudaMemsetAsync(qual, 0, size_t(c), s));
        {
            ProfScope ps(PK_OVERLAP_COLLECT, double(c) * 21, s);
            rs.epoch++;
            k_ov_hit_runs<SaT, StT><<<unsigned(ct), kScanThreads, 0, s>>>(d_sa, hits, c, d_seq_starts, nseq, run, qual,
                                                               n_runs, rs.lookback, rs.tile_ctr, rs.tile_base,
                                                               rs.epoch, status);
            LOR_LAUNCH_CHECK();
            rs.tile_base += (unsigned long long)ct;
            rs.epoch++;
            k_ov_hit_members<SaT><<<unsigned(ct), kScanThreads, 0, s>>>(d_sa, hits, c, run, qual, ka, count,
                                                                  rs.lookback, rs.tile_ctr, rs.tile_base,
                                                                  rs.epoch, status, ct);
            LOR_LAUNCH_CHECK();
            rs.tile_base += (unsigned long long)ct;
        }
        LOR_CUDA_TRY(cudaMemcpyAsync(&h_count, count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        LOR_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        LOR_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(uint32_t), s));
    }
    const int64_t m = int64_t(h_count);
    uint32_t *kr = ka, *vr = va;
    if (m > 1) {
        const int bits = bit_width_u64(uint64_t(n - 1));
        const int rc = radix_sort_pairs<uint32_t>(rs, ka, va, kb, vb, m, 0, bits, true, &kr, &vr);
        if (rc) return rc;
    }
    k_ov_result<SaT, StT, OutT><<<1, 256, 0, s>>>(d_sa, d_seq_starts, nseq, best, count, d_out);
    LOR_LAUNCH_CHECK();
    const int64_t ncopy = m < pos_cap ? m : pos_cap;
    if (ncopy > 0) {
        k_copy_u32<PosT><<<unsigned(cdiv(ncopy, 256)), 256, 0, s>>>(kr, d_pos, ncopy);
        LOR_LAUNCH_CHECK();
    }
    return LOR_OK;
}

}  // namespace
}  // namespace lor

extern "C" int lor_longest_overlap(const int32_t *d_sa, const int32_t *d_lcp, int64_t n,
                                   const int32_t *d_seq_starts, int32_t nseq, lor_overlap *d_out,
                                   int32_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                                   lor_stream_t stream) {
    return longest_overlap_impl(d_sa, d_lcp, n, d_seq_starts, nseq, d_out, d_pos, pos_cap, d_ws, ws_bytes, stream,
                                LOR_MAX_N);
}

extern "C" size_t lor_longest_overlap64_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N64) return 0;
    return ov_layout(n).total;
}

extern "C" int lor_longest_overlap64(const int64_t *d_sa, const int32_t *d_lcp, int64_t n,
                                     const int64_t *d_seq_starts, int32_t nseq, lor_overlap64 *d_out,
                                     int64_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                                     lor_stream_t stream) {
    return longest_overlap_impl(d_sa, d_lcp, n, d_seq_starts, nseq, d_out, d_pos, pos_cap, d_ws, ws_bytes, stream,
                                LOR_MAX_N64);
}
