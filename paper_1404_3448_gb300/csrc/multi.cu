// multi.cu -- one reference against many query sequences (the paper's
// experiments run 512 .. 2,097,152 query sequences against a reference;
// Section 3 defines the overlap of two sequences by their suffixes' common
// prefixes).
//
// For every query Q_i this finds the longest substring it shares with the
// reference R: L_i, the smallest offset q_i in Q_i where a length-L_i match
// starts, and the smallest offset r_i in R where Q_i[q_i, q_i + L_i) occurs.
// One suffix array covers T = R t_R Q_1 t_Q Q_2 t_Q ... with t_R = 1 (once)
// and t_Q = 2 (after every query): the common prefix of an R-suffix and a
// Q-suffix stops at the end of R (code 1 occurs once) or of the query (code
// 2 never occurs inside R), so it is a common substring of R and that query.
// The longest match of a query suffix y against R is its LCP with the nearest
// R-suffix above or below it in suffix order: the minimum of the LCP array
// between the two ranks.  So:
//   1. ranks of R-suffixes in order (Rlist) and, for every other rank, the
//      number of R-suffixes before it (one look-back scan);
//   2. per query suffix, the range minimum to the nearest R-suffix on either
//      side (block RMQ over the LCP array), kept per query as the maximum of
//      (L << 32 | ~q) by atomicMax;
//   3. per query with L > 0, the rank interval around y where the LCP stays
//      >= L (searched with the block table) and the minimum R position in it
//      (block RMQ over SA restricted to R-suffixes).
#include <climits>
#include <vector>

#include "batch.cuh"
#include "rmq_block.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_multi)

namespace lor {
namespace {

__device__ __forceinline__ int mq_seq(const int32_t *st, int nseq, int64_t p) {
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (st[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Text: sequence 0 is the reference (terminator 1), sequences 1.. are the
// queries (terminator 2); A, C, G, T (either case) -> 3..6.  starts[s] is the
// text offset of sequence s, whose ASCII bytes begin at starts[s] - s.
__global__ void k_mq_encode(const uint8_t *__restrict__ ascii, const int32_t *__restrict__ starts, int nseq,
                            int64_t n, uint8_t *__restrict__ text, int *status) {
    bool bad = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * 16;
    for (int64_t x0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 16; x0 < n; x0 += stride) {
        int q = mq_seq(starts, nseq, x0);
        for (int64_t x = x0; x < x0 + 16 && x < n; ++x) {
            while (q + 1 < nseq && x >= starts[q + 1]) ++q;
            uint8_t c;
            if (x == starts[q + 1] - 1) {
                c = q == 0 ? 1 : 2;
            } else {
                switch (ascii[x - q]) {
                    case 'A': case 'a': c = 3; break;
                    case 'C': case 'c': c = 4; break;
                    case 'G': case 'g': c = 5; break;
                    case 'T': case 't': c = 6; break;
                    default: c = 3; bad = true;
                }
            }
            text[x] = c;
        }
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
}

// Rlist[j] = rank of the j-th R-suffix (SA[k] < rlen); before[k] = number of
// R-suffixes at ranks below k; *nR = their count.  M[k] = SA[k] for
// R-suffixes, INT_MAX otherwise (the input of the position table).
__global__ void __launch_bounds__(kScanThreads) k_mq_rindex(const int32_t *__restrict__ sa, int64_t n, int64_t rlen,
                                                            int32_t *__restrict__ Rlist, int32_t *__restrict__ before,
                                                            int32_t *__restrict__ M, uint32_t *nR, uint64_t *lb,
                                                            unsigned long long *ctr, unsigned long long tile_base,
                                                            uint32_t epoch, int *status, int64_t ntiles) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    int32_t v[kScanItems];
    load_run<int32_t, kScanItems>(sa, base, n, -1, v);
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const bool r = base + i < n && v[i] >= 0 && v[i] < rlen;
        flags |= uint32_t(r) << i;
        cnt += r ? 1u : 0u;
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) {
            s_prefix = p;
            if (tile == ntiles - 1) *nR = p + agg;
        }
    }
    __syncthreads();
    uint32_t o = s_prefix + excl;
    int32_t bf[kScanItems], mm[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const bool r = (flags >> i) & 1u;
        bf[i] = int32_t(o);
        mm[i] = r ? v[i] : INT_MAX;
        if (r) Rlist[o++] = int32_t(base + i);
    }
    store_run<int32_t, kScanItems>(before, base, n, bf);
    store_run<int32_t, kScanItems>(M, base, n, mm);
}

// Per query suffix: its longest match in R, folded into best[query].
__global__ void k_mq_best(const uint8_t *__restrict__ text, const int32_t *__restrict__ sa,
                          const int32_t *__restrict__ lcp, int64_t n, int64_t rlen, const int32_t *__restrict__ table,
                          int64_t stride, const int32_t *__restrict__ Rlist, const int32_t *__restrict__ before,
                          const uint32_t *nR_dev, const int32_t *__restrict__ starts, int nseq,
                          unsigned long long *__restrict__ best) {
    const int64_t nR = int64_t(*nR_dev);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int32_t y = sa[k];
        if (y <= rlen || y >= n || text[y] < 3) continue;  // R, its terminator, a query terminator
        const int64_t j = before[k];
        int32_t up = 0, down = 0;
        if (j > 0) up = rmqb_range_min(table, stride, lcp, int64_t(Rlist[j - 1]) + 1, k);
        if (j < nR) down = rmqb_range_min(table, stride, lcp, k + 1, Rlist[j]);
        const int32_t L = max(up, down);
        if (L <= 0) continue;
        const int s = mq_seq(starts, nseq, y);
        const uint32_t q = uint32_t(y - starts[s]);
        atomicMax(&best[s - 1], (static_cast<unsigned long long>(uint32_t(L)) << 32) | (0xFFFFFFFFull - q));
    }
}

// Last rank k' <= k with lcp[k'] < L (lcp[0] = 0 < L, so one exists).
__device__ int64_t mq_left(const int32_t *__restrict__ lcp, const int32_t *__restrict__ table, int64_t stride,
                           int levels, int64_t k, int32_t L) {
    const int64_t bk = k / kRmqBlock;
    for (int64_t i = k; i >= bk * kRmqBlock; --i)
        if (lcp[i] < L) return i;
    int64_t pos = bk - 1;  // last block that may hold a value < L
    for (int j = levels - 1; j >= 0; --j) {
        const int64_t w = int64_t(1) << j;
        if (pos - w + 1 >= 0 && table[int64_t(j) * stride + pos - w + 1] >= L) pos -= w;
    }
    if (pos < 0) return 0;
    for (int64_t i = pos * kRmqBlock + kRmqBlock - 1; i >= pos * kRmqBlock; --i)
        if (lcp[i] < L) return i;
    return 0;
}

// First rank k'' > k with lcp[k''] < L, or n.
__device__ int64_t mq_right(const int32_t *__restrict__ lcp, const int32_t *__restrict__ table, int64_t stride,
                            int levels, int64_t nb, int64_t n, int64_t k, int32_t L) {
    const int64_t bk = k / kRmqBlock;
    const int64_t bend = min64(bk * kRmqBlock + kRmqBlock, n);
    for (int64_t i = k + 1; i < bend; ++i)
        if (lcp[i] < L) return i;
    int64_t pos = bk + 1;  // first block that may hold a value < L
    for (int j = levels - 1; j >= 0; --j) {
        const int64_t w = int64_t(1) << j;
        if (pos + w - 1 < nb && table[int64_t(j) * stride + pos] >= L) pos += w;
    }
    if (pos >= nb) return n;
    const int64_t e = min64(pos * kRmqBlock + kRmqBlock, n);
    for (int64_t i = pos * kRmqBlock; i < e; ++i)
        if (lcp[i] < L) return i;
    return n;
}

__global__ void k_mq_result(const unsigned long long *__restrict__ best, int nq, const int32_t *__restrict__ starts,
                            const int32_t *__restrict__ isa, const int32_t *__restrict__ lcp,
                            const int32_t *__restrict__ table, const int32_t *__restrict__ mtab, int64_t stride,
                            int levels, const int32_t *__restrict__ M, int64_t n, lor_mq_hit *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const unsigned long long b = best[i];
    lor_mq_hit h;
    h.reserved = 0;
    const int32_t L = int32_t(b >> 32);
    if (L <= 0) {
        h.length = 0;
        h.query_pos = h.ref_pos = -1;
    } else {
        const int32_t q = int32_t(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
        const int64_t k = isa[int64_t(starts[i + 1]) + q];
        const int64_t lo = mq_left(lcp, table, stride, levels, k, L);
        const int64_t hi = mq_right(lcp, table, stride, levels, rmqb_blocks(n), n, k, L) - 1;
        h.length = L;
        h.query_pos = q;
        h.ref_pos = rmqb_range_min(mtab, stride, M, lo, hi);
    }
    out[i] = h;
}

struct MqLayout {
    size_t text = 0, starts = 0, sa = 0, isa = 0, lcp = 0, region = 0, total = 0;
    // inside the region, once the suffix array and the LCP array are built
    size_t ctrl = 0, lookback = 0, lookback_bytes = 0, rlist = 0, before = 0, M = 0, table = 0, mtab = 0,
           best = 0, post = 0;
    int levels = 0;
    int64_t stride = 0;
};

MqLayout mq_layout(int64_t n, int nq) {
    MqLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.text = take(size_t(n));
    L.starts = take(sizeof(int32_t) * (size_t(nq) + 2));
    L.sa = take(sizeof(int32_t) * size_t(n));
    L.isa = take(sizeof(int32_t) * size_t(n));
    L.lcp = take(sizeof(int32_t) * size_t(n));
    L.region = off;
    size_t r = 0;
    auto rtake = [&](size_t bytes) {
        size_t o = r;
        r = align256(r + bytes);
        return L.region + o;
    };
    const int64_t nb = rmqb_blocks(n);
    L.levels = bit_width_u64(uint64_t(nb));
    L.stride = rmq_row_stride_of(nb);
    L.ctrl = rtake(256);
    L.lookback_bytes = sizeof(uint64_t) * size_t(cdiv(n, kScanTile));
    L.lookback = rtake(L.lookback_bytes);
    L.rlist = rtake(sizeof(int32_t) * size_t(n));
    L.before = rtake(sizeof(int32_t) * size_t(n));
    L.M = rtake(sizeof(int32_t) * size_t(n));
    L.table = rtake(sizeof(int32_t) * size_t(L.levels) * size_t(L.stride));
    L.mtab = rtake(sizeof(int32_t) * size_t(L.levels) * size_t(L.stride));
    L.best = rtake(sizeof(unsigned long long) * size_t(nq > 0 ? nq : 1));
    L.post = r;
    size_t need = L.post;
    const size_t sa_ws = lor_build_sa_workspace_size(n, 7), lcp_ws = lor_lcp_workspace_size(n);
    need = sa_ws > need ? sa_ws : need;
    need = lcp_ws > need ? lcp_ws : need;
    L.total = L.region + need;
    return L;
}

bool mq_sizes(int64_t ref_len, const int64_t *h_q_lens, int32_t nq, int64_t *n) {
    if (ref_len < 0 || nq < 1 || !h_q_lens || nq > LOR_MQ_MAX_QUERIES) return false;
    int64_t t = ref_len + 1;
    for (int i = 0; i < nq; ++i) {
        if (h_q_lens[i] < 0) return false;
        t += h_q_lens[i] + 1;
        if (t > LOR_MAX_N) return false;
    }
    *n = t;
    return true;
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_multi_query_workspace_size(int64_t ref_len, const int64_t *h_q_lens, int32_t nq) {
    int64_t n = 0;
    if (!mq_sizes(ref_len, h_q_lens, nq, &n)) return 0;
    return mq_layout(n, nq).total;
}

extern "C" int lor_multi_query_overlap(const uint8_t *d_ref, int64_t ref_len, const uint8_t *d_queries,
                                       const int64_t *h_q_lens, int32_t nq, lor_mq_hit *d_out, void *d_ws,
                                       size_t ws_bytes, lor_stream_t stream) {
    int64_t n = 0;
    if (!d_out || !h_q_lens || nq < 1 || ref_len < 0) return LOR_ERR_INVALID_ARG;
    if (nq > LOR_MQ_MAX_QUERIES) return LOR_ERR_TOO_LARGE;
    if (!mq_sizes(ref_len, h_q_lens, nq, &n)) {
        for (int i = 0; i < nq; ++i)
            if (h_q_lens[i] < 0) return LOR_ERR_INVALID_ARG;
        return LOR_ERR_TOO_LARGE;
    }
    int64_t qtotal = 0;
    for (int i = 0; i < nq; ++i) qtotal += h_q_lens[i];
    if ((ref_len > 0 && !d_ref) || (qtotal > 0 && !d_queries)) return LOR_ERR_INVALID_ARG;
    const MqLayout L = mq_layout(n, nq);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    char *ws = (char *)d_ws;
    uint8_t *text = (uint8_t *)(ws + L.text);
    int32_t *starts = (int32_t *)(ws + L.starts);
    int32_t *sa = (int32_t *)(ws + L.sa), *isa = (int32_t *)(ws + L.isa), *lcp = (int32_t *)(ws + L.lcp);
    const int nseq = nq + 1;
    // The reference and the queries go to the device back to back: the
    // reference's bytes first, then every query's, at ascii offset starts[s] - s.
    {
        std::vector<int32_t> hst(size_t(nseq) + 1);
        int64_t x = 0;
        hst[0] = 0;
        x = ref_len + 1;
        for (int i = 0; i < nq; ++i) {
            hst[size_t(i) + 1] = int32_t(x);
            x += h_q_lens[i] + 1;
        }
        hst[size_t(nseq)] = int32_t(x);
        // pageable source: the copy has left hst when the call returns
        LOR_CUDA_TRY(cudaMemcpyAsync(starts, hst.data(), sizeof(int32_t) * hst.size(), cudaMemcpyHostToDevice, s));
    }
    // The encode kernel reads sequence s's bases at starts[s] - s of one
    // ASCII buffer: stage the reference right before the queries.
    uint8_t *ascii = (uint8_t *)(ws + L.region);
    if (ref_len > 0)
        LOR_CUDA_TRY(cudaMemcpyAsync(ascii, d_ref, size_t(ref_len), cudaMemcpyDeviceToDevice, s));
    if (qtotal > 0)
        LOR_CUDA_TRY(cudaMemcpyAsync(ascii + ref_len, d_queries, size_t(qtotal), cudaMemcpyDeviceToDevice, s));
    {
        ProfScope ps(PK_ENCODE, double(n) * 2, s);
        k_mq_encode<<<unsigned(min64(cdiv(cdiv(n, 16), 256), 152 * 8)), 256, 0, s>>>(ascii, starts, nseq, n, text,
                                                                                     status);
    }
    LOR_LAUNCH_CHECK();
    int rc = build_sa_impl(text, n, 7, sa, ws + L.region, ws_bytes - L.region, s, nullptr, 0);
    if (rc) return rc;
    rc = lor_lcp(text, sa, n, isa, lcp, ws + L.region, ws_bytes - L.region, (lor_stream_t)s);
    if (rc) return rc;
    // post-processing buffers reuse the region
    unsigned long long *ctr = (unsigned long long *)(ws + L.ctrl);
    uint32_t *nR = (uint32_t *)(ws + L.ctrl + 64);
    uint64_t *lb = (uint64_t *)(ws + L.lookback);
    int32_t *Rlist = (int32_t *)(ws + L.rlist), *before = (int32_t *)(ws + L.before), *M = (int32_t *)(ws + L.M);
    int32_t *table = (int32_t *)(ws + L.table), *mtab = (int32_t *)(ws + L.mtab);
    unsigned long long *best = (unsigned long long *)(ws + L.best);
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(lb, 0, L.lookback_bytes, s));
    LOR_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long) * size_t(nq), s));
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 16, s);
        const int64_t ntiles = cdiv(n, kScanTile);
        k_mq_rindex<<<unsigned(ntiles), kScanThreads, 0, s>>>(sa, n, ref_len, Rlist, before, M, nR, lb, ctr, 0, 1,
                                                             status, ntiles);
    }
    LOR_LAUNCH_CHECK();
    rc = rmq_block_levels(lcp, n, L.levels, table, s);
    if (rc) return rc;
    rc = rmq_block_levels(M, n, L.levels, mtab, s);
    if (rc) return rc;
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 24, s);
        k_mq_best<<<unsigned(min64(cdiv(n, 256), 152 * 16)), 256, 0, s>>>(text, sa, lcp, n, ref_len, table,
                                                                         L.stride, Rlist, before, nR, starts, nseq,
                                                                         best);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(nq) * 64, s);
        k_mq_result<<<unsigned(cdiv(nq, 128)), 128, 0, s>>>(best, nq, starts, isa, lcp, table, mtab, L.stride,
                                                           L.levels, M, n, d_out);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
