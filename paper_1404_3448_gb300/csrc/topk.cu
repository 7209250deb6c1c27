// topk.cu -- the K longest maximal overlaps between different sequences
// (extends the longest overlap of Section 3 from the maximum to the K
// largest values of the same quantity).
//
// A candidate is a rank k whose adjacent suffixes a = SA[k-1], b = SA[k]
// come from different sequences, with LCP[k] > 0, and that is left-maximal:
// a or b starts the text, or the symbols before a and b differ (a suffix
// starting a sequence is preceded by the previous sequence's own terminator,
// so it always counts as different).  Left-maximality keeps one candidate
// per shared region instead of one per shifted copy of it.  The K largest
// candidates by (LCP desc, rank asc) are reported, each as an overlap record
// (the first equals lor_longest_overlap's record whenever that one is
// left-maximal).
//
// Selection without host round trips: a 4096-bin histogram of min(LCP, 4095)
// over the candidates gives the threshold t (the largest value with at least
// K candidates at LCP >= t, or 1 when there are fewer than K); the candidates
// with LCP >= t are compacted, radix sorted by (LCP desc, rank asc) with the
// count read from device memory, and the first K emitted.
#include "radix.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_topk)

namespace lor {
namespace {

constexpr int kTopkBins = 4096;

__device__ __forceinline__ int tk_seq(const int32_t *starts, int nseq, int32_t p) {
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool tk_candidate(const uint8_t *text, const int32_t *sa, const int32_t *lcp,
                                             const int32_t *sst, int nseq, int64_t k) {
    if (k < 1 || lcp[k] <= 0) return false;
    const int32_t a = sa[k - 1], b = sa[k];
    if (a != 0 && b != 0 && text[a - 1] == text[b - 1]) return false;
    return tk_seq(sst, nseq, a) != tk_seq(sst, nseq, b);
}

__global__ void __launch_bounds__(256) k_topk_hist(const uint8_t *__restrict__ text, const int32_t *__restrict__ sa,
                                                   const int32_t *__restrict__ lcp, int64_t n,
                                                   const int32_t *__restrict__ starts, int nseq,
                                                   uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[kTopkBins];
    __shared__ int32_t sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x) sh[i] = 0;
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        if (tk_candidate(text, sa, lcp, sst, nseq, k)) atomicAdd(&sh[min(lcp[k], kTopkBins - 1)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One thread: the threshold (see the file comment) into *thr.
__global__ void k_topk_threshold(const uint32_t *__restrict__ hist, int K, int32_t *thr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t cum = 0;
    int t = 1;
    for (int b = kTopkBins - 1; b >= 1; --b) {
        cum += hist[b];
        if (cum >= uint64_t(K)) {
            t = b;
            break;
        }
    }
    *thr = t;
}

// Sort key (2^31 - 1 - LCP) << 32 | rank: ascending = LCP desc, rank asc.
__global__ void __launch_bounds__(kScanThreads) k_topk_compact(const uint8_t *__restrict__ text,
                                                               const int32_t *__restrict__ sa,
                                                               const int32_t *__restrict__ lcp, int64_t n,
                                                               const int32_t *__restrict__ starts, int nseq,
                                                               const int32_t *thr, uint64_t *__restrict__ keys,
                                                               uint32_t *count, uint64_t *lb, unsigned long long *ctr,
                                                               unsigned long long tile_base, uint32_t epoch,
                                                               int *status, int64_t ntiles) {
    __shared__ int32_t sst[LOR_MAX_SEQ + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    const int32_t t = *thr;
    tile_compact(
        n, [&](int64_t k) { return lcp[k] >= t && tk_candidate(text, sa, lcp, sst, nseq, k); },
        [&](int64_t k, uint32_t o) {
            keys[o] = (uint64_t(uint32_t(0x7FFFFFFF - lcp[k])) << 32) | uint64_t(uint32_t(k));
        },
        lb, ctr, tile_base, epoch, status, count, ntiles);
}

__global__ void k_topk_emit(const uint64_t *__restrict__ keys, const uint32_t *count, int K,
                            const int32_t *__restrict__ sa, const int32_t *__restrict__ starts, int nseq,
                            lor_overlap *__restrict__ out, int32_t *n_out) {
    const int64_t c = int64_t(*count);
    const int kk = int(c < K ? c : K);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *n_out = kk;
    if (i >= kk) return;
    const uint64_t key = keys[i];
    const int64_t k = int64_t(uint32_t(key));
    int32_t a = sa[k - 1], b = sa[k];
    int qa = tk_seq(starts, nseq, a), qb = tk_seq(starts, nseq, b);
    if (qa > qb) {
        const int32_t t = a; a = b; b = t;
        const int u = qa; qa = qb; qb = u;
    }
    lor_overlap r;
    r.length = 0x7FFFFFFF - int32_t(key >> 32);
    r.rank = int32_t(k);
    r.seq_a = qa;
    r.pos_a = a - starts[qa];
    r.seq_b = qb;
    r.pos_b = b - starts[qb];
    r.n_pos = 0;
    r.reserved = 0;
    out[i] = r;
}

struct TkLayout {
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0, thr = 0, k0 = 0, k1 = 0, v0 = 0,
           v1 = 0, total = 0;
};

TkLayout tk_layout(int64_t n) {
    TkLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * (kMaxPasses * kRadix > kTopkBins ? kMaxPasses * kRadix : kTopkBins));
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(n);
    L.lookback = take(L.lookback_bytes);
    L.thr = take(sizeof(int32_t));
    L.k0 = take(sizeof(uint64_t) * size_t(n));
    L.k1 = take(sizeof(uint64_t) * size_t(n));
    L.v0 = take(sizeof(uint32_t) * size_t(n));
    L.v1 = take(sizeof(uint32_t) * size_t(n));
    L.total = off;
    return L;
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_topk_overlaps_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return tk_layout(n).total;
}

extern "C" int lor_topk_overlaps(const uint8_t *d_text, const int32_t *d_sa, const int32_t *d_lcp, int64_t n,
                                 const int32_t *d_seq_starts, int32_t nseq, int32_t K, lor_overlap *d_out,
                                 int32_t *d_count, void *d_ws, size_t ws_bytes, lor_stream_t stream) {
    if (!d_text || !d_sa || !d_lcp || !d_seq_starts || !d_out || !d_count || n < 1) return LOR_ERR_INVALID_ARG;
    if (nseq < 1 || nseq > LOR_MAX_SEQ || K < 1 || K > LOR_TOPK_MAX) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const TkLayout L = tk_layout(n);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    char *ws = (char *)d_ws;
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl);
    rs.max_tiles = cdiv(n, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    uint32_t *count = (uint32_t *)(ws + L.ctrl + 128);
    int32_t *thr = (int32_t *)(ws + L.thr);
    uint64_t *k0 = (uint64_t *)(ws + L.k0), *k1 = (uint64_t *)(ws + L.k1);
    uint32_t *v0 = (uint32_t *)(ws + L.v0), *v1 = (uint32_t *)(ws + L.v1);
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    LOR_CUDA_TRY(cudaMemsetAsync(rs.hist, 0, sizeof(uint32_t) * kTopkBins, s));
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 10, s);
        k_topk_hist<<<unsigned(min64(cdiv(n, 256), 152 * 8)), 256, 0, s>>>(d_text, d_sa, d_lcp, n, d_seq_starts, nseq,
                                                                           rs.hist);
        LOR_LAUNCH_CHECK();
        k_topk_threshold<<<1, 32, 0, s>>>(rs.hist, K, thr);
        LOR_LAUNCH_CHECK();
    }
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 10, s);
        const int64_t ntiles = cdiv(n, kScanTile);
        rs.epoch++;
        k_topk_compact<<<unsigned(ntiles), kScanThreads, 0, s>>>(d_text, d_sa, d_lcp, n, d_seq_starts, nseq, thr, k0,
                                                                 count, rs.lookback, rs.tile_ctr, rs.tile_base,
                                                                 rs.epoch, status, ntiles);
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
    }
    uint64_t *kr;
    uint32_t *vr;
    int rc = radix_sort_pairs<uint64_t>(rs, k0, v0, k1, v1, n, 0, 63, true, &kr, &vr, false, count);
    if (rc) return rc;
    k_topk_emit<<<unsigned(cdiv(K, 128)), 128, 0, s>>>(kr, count, K, d_sa, d_seq_starts, nseq, d_out, d_count);
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
