// batch.cu -- longest overlap region of many sequence pairs at once.
//
// Pairs are processed in groups of up to 512 pairs and 2^28 symbols.  The
// group text is the concatenation of every pair's own text S1#S2$ with the
// codes of a two-sequence text ($ = 1 < # = 2 < A < C < G < T), so the
// terminator codes repeat from pair to pair.  One suffix array is built over
// the group text with the DC3 of lor_build_sa; a stable radix sort on the
// pair id then splits it into one block per pair.  Two suffixes of the same
// pair are decided at the latest where the first of them reaches its own
// terminator: at that offset the other holds a base or the other terminator,
// exactly as in the pair's own text, so the order never depends on what
// follows a terminator and block p is the suffix array of pair p's S1#S2$
// (shifted by the pair's offset in the group text).  The LCP inside the blocks comes from the
// Kasai kernels with the predecessor of every block head cleared, and the
// overlap is the segmented form of lor_longest_overlap (Section 3): one
// argmax per block, runs with LCP >= L_p inside blocks, members compacted and
// sorted.  Every pair's record and positions equal those of lor_longest_overlap
// run on that pair alone.
#include <algorithm>
#include <vector>

#include "batch.cuh"
#include "lcp_kernels.cuh"
#include "radix.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_batch)

namespace lor {
namespace {

__device__ __forceinline__ int bseq(const int32_t *st, int nseq, int32_t p) {
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (st[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_pair_keys(const int32_t *__restrict__ sa, int64_t n, const int32_t *__restrict__ starts,
                            int nseq, uint32_t *__restrict__ key) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        key[k] = uint32_t(bseq(sst, nseq, sa[k]) >> 1);
}

__global__ void k_block_starts(const uint32_t *__restrict__ pk, int64_t n, int32_t *__restrict__ bstart) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < n && (k == 0 || pk[k] != pk[k - 1])) bstart[pk[k]] = int32_t(k);
}

// best[p] = max over block p of (LCP[k] << 32 | ~(k - block start)) for ranks
// k whose neighbour k-1 in the block starts in the other sequence.
__global__ void __launch_bounds__(256) k_seg_argmax(const int32_t *__restrict__ sa,
                                                    const int32_t *__restrict__ lcp,
                                                    const uint32_t *__restrict__ pk, int64_t n,
                                                    const int32_t *__restrict__ bstart,
                                                    const int32_t *__restrict__ starts, int nseq,
                                                    unsigned long long *best) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const int64_t k = base + threadIdx.x;
        unsigned long long key = 0;
        uint32_t p = 0xFFFFFFFFu;
        if (k < n) {
            p = pk[k];
            const int64_t b = bstart[p];
            if (k > b && bseq(sst, nseq, sa[k - 1]) != bseq(sst, nseq, sa[k]))
                key = (static_cast<unsigned long long>(uint32_t(lcp[k])) << 32) |
                      (0xFFFFFFFFull - uint64_t(k - b));
        }
        const uint32_t p0 = __shfl_sync(0xffffffffu, p, 0);
        if (__all_sync(0xffffffffu, p == p0)) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
                key = o > key ? o : key;
            }
            if ((threadIdx.x & 31) == 0 && key && p0 != 0xFFFFFFFFu) atomicMax(&best[p0], key);
        } else if (key) {
            atomicMax(&best[p], key);
        }
    }
}

__device__ __forceinline__ bool seg_run_start(int64_t k, const uint32_t *pk, const int32_t *bstart,
                                              const int32_t *lcp, const unsigned long long *best) {
    const uint32_t p = pk[k];
    const int32_t L = int32_t(best[p] >> 32);
    return k == bstart[p] || L <= 0 || lcp[k] < L;
}

__global__ void __launch_bounds__(kScanThreads) k_seg_runs(const uint32_t *__restrict__ pk,
                                                           const int32_t *__restrict__ bstart,
                                                           const int32_t *__restrict__ lcp,
                                                           const unsigned long long *__restrict__ best,
                                                           int64_t n, int32_t *__restrict__ run_id,
                                                           uint32_t *n_runs, uint64_t *lb,
                                                           unsigned long long *ctr,
                                                           unsigned long long tile_base, uint32_t epoch,
                                                           int *status) {
    tile_names(
        n, [&](int64_t k) { return seg_run_start(k, pk, bstart, lcp, best); },
        [&](int64_t k, uint32_t name) { run_id[k] = int32_t(name) - 1; }, n_runs, lb, ctr, tile_base,
        epoch, status);
}

__global__ void k_seg_qual(const int32_t *__restrict__ sa, const uint32_t *__restrict__ pk,
                           const int32_t *__restrict__ bstart, const int32_t *__restrict__ lcp,
                           const unsigned long long *__restrict__ best, int64_t n,
                           const int32_t *__restrict__ starts, int nseq, const int32_t *__restrict__ run_id,
                           uint8_t *__restrict__ qual) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        if (seg_run_start(k, pk, bstart, lcp, best)) continue;
        if (bseq(sst, nseq, sa[k - 1]) != bseq(sst, nseq, sa[k])) qual[run_id[k]] = 1;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_seg_members(
    const int32_t *__restrict__ sa, int64_t n, const int32_t *__restrict__ run_id,
    const uint8_t *__restrict__ qual, uint32_t *__restrict__ out, uint32_t *count, uint64_t *lb,
    unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch, int *status, int64_t ntiles) {
    tile_compact(
        n, [&](int64_t k) { return qual[run_id[k]] != 0; },
        [&](int64_t k, uint32_t o) { out[o] = uint32_t(sa[k]); }, lb, ctr, tile_base, epoch, status, count,
        ntiles);
}

// m_dev (when given) holds the member count on the device.
__global__ void k_pair_count(const uint32_t *__restrict__ pos, int64_t m, const uint32_t *m_dev,
                             const int32_t *__restrict__ starts, int nseq, int32_t *__restrict__ cnt) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    if (m_dev) m = int64_t(*m_dev);
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[bseq(sst, nseq, int32_t(pos[i])) >> 1], 1);
}

// One block: records and position offsets of the group's pairs.
// pos_base_dev (when given) holds the group's first position slot on the
// device.
__global__ void k_group_finish(const int32_t *__restrict__ sa, const int32_t *__restrict__ bstart,
                               const unsigned long long *__restrict__ best, const int32_t *__restrict__ cnt,
                               const int32_t *__restrict__ starts, int nseq, int npairs, int64_t pos_base,
                               const int64_t *pos_base_dev, lor_overlap *__restrict__ out,
                               int64_t *__restrict__ pos_off) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    __shared__ int64_t soff[kPairsPerGroup + 1];
    if (pos_base_dev) pos_base = *pos_base_dev;
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int p = 0; p < npairs; ++p) {
            soff[p] = acc;
            acc += cnt[p];
        }
        soff[npairs] = acc;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        lor_overlap r;
        r.reserved = 0;
        const unsigned long long b = best[p];
        const int32_t L = int32_t(b >> 32);
        if (L <= 0) {
            r.length = 0;
            r.rank = r.seq_a = r.pos_a = r.seq_b = r.pos_b = -1;
            r.n_pos = 0;
        } else {
            const int64_t k0 = bstart[p];
            const int64_t k = k0 + int64_t(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
            int32_t a = sa[k - 1], c = sa[k];
            int qa = bseq(sst, nseq, a), qc = bseq(sst, nseq, c);
            if (qa > qc) {
                const int32_t t = a; a = c; c = t;
                const int u = qa; qa = qc; qc = u;
            }
            r.length = L;
            r.rank = int32_t(k - k0);
            r.seq_a = qa - 2 * p;
            r.pos_a = a - sst[qa];
            r.seq_b = qc - 2 * p;
            r.pos_b = c - sst[qc];
            r.n_pos = cnt[p];
        }
        out[p] = r;
        pos_off[p] = pos_base + soff[p];
    }
    if (threadIdx.x == 0) pos_off[npairs] = pos_base + soff[npairs];
}

// Positions sorted by text position are grouped by pair, in pair order: the
// i-th goes to slot pos_base + i, as an offset inside its pair's own text.
__global__ void k_group_positions(const uint32_t *__restrict__ pos, int64_t m, const uint32_t *m_dev,
                                  const int32_t *__restrict__ starts, int nseq, int64_t pos_base,
                                  const int64_t *pos_base_dev, int32_t *__restrict__ dst, int64_t cap) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    if (m_dev) m = int64_t(*m_dev);
    if (pos_base_dev) pos_base = *pos_base_dev;
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m && pos_base + i < cap;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t x = int32_t(pos[i]);
        const int pair = bseq(sst, nseq, x) >> 1;
        dst[pos_base + i] = x - sst[2 * pair];
    }
}

// The next group's first position slot: this group's plus its count.
__global__ void k_group_pos_advance(int64_t *pos_base_dev, const uint32_t *m_dev) {
    if (threadIdx.x == 0) *pos_base_dev += int64_t(*m_dev);
}

// Group text: sequence q's bases (ASCII ACGT/acgt -> 3..6) followed by its
// terminator (# = 2 after the first sequence of a pair, $ = 1 after the
// second).  starts[q] is where sequence q begins in the text; its ASCII bytes
// begin at starts[q] - q.  Each thread writes 16 consecutive symbols.
__global__ void k_encode_group(const uint8_t *__restrict__ ascii, const int32_t *__restrict__ starts, int nseq,
                               int64_t n, uint8_t *__restrict__ text, int *status) {
    __shared__ int32_t sst[kGroupSeqs + 1];
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) sst[i] = starts[i];
    __syncthreads();
    bool bad = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * 16;
    for (int64_t x0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 16; x0 < n; x0 += stride) {
        int q = bseq(sst, nseq, int32_t(x0));
        for (int64_t x = x0; x < x0 + 16 && x < n; ++x) {
            while (q + 1 < nseq && x >= sst[q + 1]) ++q;
            uint8_t c;
            if (x == sst[q + 1] - 1) {
                c = (q & 1) ? 1 : 2;
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

struct Group {
    int p0, np;     // first pair, pair count
    int64_t in0;    // offset of its first ASCII byte
    int64_t n;      // text length
};

std::vector<Group> make_groups(const int64_t *lens, int npairs) {
    std::vector<Group> g;
    int64_t in = 0;
    int p = 0;
    while (p < npairs) {
        Group cur{p, 0, in, 0};
        while (p < npairs && cur.np < kPairsPerGroup) {
            const int64_t add = lens[2 * p] + lens[2 * p + 1] + 2;
            if (cur.np > 0 && cur.n + add > kGroupSymbolCap) break;
            cur.n += add;
            in += lens[2 * p] + lens[2 * p + 1];
            ++cur.np;
            ++p;
        }
        g.push_back(cur);
    }
    return g;
}

}  // namespace

BatchLayout batch_layout(int64_t nmax) {
    BatchLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.text = take(size_t(nmax));
    L.starts = take(sizeof(int32_t) * (kGroupSeqs + 1));
    L.sa = take(sizeof(int32_t) * size_t(nmax));
    L.region = off;
    size_t r = 0;
    auto rtake = [&](size_t bytes) {
        size_t o = r;
        r = align256(r + bytes);
        return L.region + o;
    };
    const size_t n4 = sizeof(int32_t) * size_t(nmax);
    L.ctrl = rtake(256);
    L.hist = rtake(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = rtake(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(nmax);
    L.lookback = rtake(L.lookback_bytes);
    L.pk = rtake(n4);
    L.pk2 = rtake(n4);
    L.sa2 = rtake(n4);
    L.ip = rtake(2 * n4);
    L.isa = rtake(n4);
    L.plcp = rtake(n4);
    L.lcp = rtake(n4);
    L.run_id = rtake(n4);
    L.qual = rtake(size_t(nmax));
    L.mem = rtake(n4);
    L.kb = rtake(n4);
    L.va = rtake(n4);
    L.vb = rtake(n4);
    L.packed = rtake(packed_text_bytes(nmax));
    L.bstart = rtake(sizeof(int32_t) * kPairsPerGroup);
    L.best = rtake(sizeof(unsigned long long) * kPairsPerGroup);
    L.cnt = rtake(sizeof(int32_t) * kPairsPerGroup);
    L.post = r;
    const size_t sa_ws = lor_build_sa_workspace_size(nmax, 7);
    L.total = L.region + (sa_ws > L.post ? sa_ws : L.post);
    return L;
}

namespace {
unsigned gridn(int64_t m, int nt) { return unsigned(cdiv(m > 0 ? m : 1, nt)); }
// Grid of the grid-stride kernels that stage the group's starts in shared
// memory first (a few blocks per SM, not one per 256 items).
unsigned gridc(int64_t m) { return unsigned(min64(cdiv(m > 0 ? m : 1, 256), 152 * 8)); }
}  // namespace

int batch_group(const uint8_t *d_ascii, const int64_t *h_lens, int np, int64_t n, char *ws, size_t ws_bytes,
                const BatchLayout &L, int64_t nmax, const GroupOutputs &o, int64_t *h_found, cudaStream_t s,
                const GroupGraph *g) {
    const int nseq = 2 * np;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    uint8_t *text = (uint8_t *)(ws + L.text);
    int32_t *starts = (int32_t *)(ws + L.starts);
    int32_t *sa = (int32_t *)(ws + L.sa);
    if (np < 1 || np > kPairsPerGroup) return LOR_ERR_INVALID_ARG;
    {
        std::vector<int32_t> hst(size_t(nseq) + 1);
        int64_t x = 0;
        for (int q = 0; q < nseq; ++q) {
            hst[q] = int32_t(x);
            x += h_lens[q] + 1;
        }
        hst[nseq] = int32_t(x);
        if (x != n) return LOR_ERR_INVALID_ARG;
        if (g) {
            // captured copy: the source must outlive the graph (pinned, owned by it)
            std::copy(hst.begin(), hst.end(), g->h_starts);
            LOR_CUDA_TRY(cudaMemcpyAsync(starts, g->h_starts, sizeof(int32_t) * hst.size(), cudaMemcpyHostToDevice, s));
        } else {
            // pageable source: the copy has left hst when the call returns
            LOR_CUDA_TRY(cudaMemcpyAsync(starts, hst.data(), sizeof(int32_t) * hst.size(), cudaMemcpyHostToDevice, s));
        }
    }
    {
        ProfScope ps(PK_ENCODE, double(n) * 2, s);
        k_encode_group<<<gridc(cdiv(n, 16)), 256, 0, s>>>(d_ascii, starts, nseq, n, text, status);
    }
    LOR_LAUNCH_CHECK();
    int rc = build_sa_impl(text, n, 7, sa, ws + L.region, ws_bytes - L.region, s, g ? g->sa_pool : nullptr,
                           g ? g->sa_pool_size : 0);
    if (rc) return rc;
    // The suffix-array workspace is free again: carve the group buffers.
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl);
    rs.max_tiles = cdiv(nmax, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    if (g) {
        rs.graph = true;
        rs.ctr_pool = g->post_pool;
        rs.ctr_pool_size = g->post_pool_size;
        LOR_CUDA_TRY(cudaMemsetAsync(g->post_pool, 0, sizeof(unsigned long long) * size_t(g->post_pool_size), s));
    }
    uint32_t *pk = (uint32_t *)(ws + L.pk), *pk2 = (uint32_t *)(ws + L.pk2);
    int32_t *sa2 = (int32_t *)(ws + L.sa2), *isa = (int32_t *)(ws + L.isa);
    int32_t *plcp = (int32_t *)(ws + L.plcp), *lcp = (int32_t *)(ws + L.lcp);
    int32_t *run_id = (int32_t *)(ws + L.run_id), *bstart = (int32_t *)(ws + L.bstart);
    int32_t *cnt = (int32_t *)(ws + L.cnt);
    uint8_t *qual = (uint8_t *)(ws + L.qual);
    uint32_t *mem = (uint32_t *)(ws + L.mem), *kb = (uint32_t *)(ws + L.kb);
    uint32_t *va = (uint32_t *)(ws + L.va), *vb = (uint32_t *)(ws + L.vb);
    unsigned long long *best = (unsigned long long *)(ws + L.best);
    uint32_t *d_count = (uint32_t *)(ws + L.ctrl + 128);
    uint32_t *d_runs = (uint32_t *)(ws + L.ctrl + 192);
    int2 *ip = (int2 *)(ws + L.ip);
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    LOR_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long) * kPairsPerGroup, s));
    LOR_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * kPairsPerGroup, s));
    LOR_CUDA_TRY(cudaMemsetAsync(qual, 0, size_t(n), s));

    // Per-pair blocks of the suffix array (stable by pair id).
    k_pair_keys<<<gridc(n), 256, 0, s>>>(sa, n, starts, nseq, pk);
    LOR_LAUNCH_CHECK();
    uint32_t *kr, *vr;
    rc = radix_sort_pairs<uint32_t>(rs, pk, (uint32_t *)sa, pk2, (uint32_t *)sa2, n, 0,
                                    bit_width_u64(uint64_t(np - 1)), false, &kr, &vr);
    if (rc) return rc;
    const uint32_t *PK = kr;
    const int32_t *SA = (const int32_t *)vr;
    k_block_starts<<<gridn(n, 256), 256, 0, s>>>(PK, n, bstart);
    LOR_LAUNCH_CHECK();

    // LCP inside the blocks.
    {
        ProfScope ps(PK_ISA_SCATTER, double(n) * 16, s);
        k_isa_phi<<<gridn(n, 256), 256, 0, s>>>(SA, n, PK, ip, status);
    }
    LOR_LAUNCH_CHECK();
    const PackedText T = packed_text_at(ws + L.packed, n);
    {
        ProfScope ps(PK_KASAI, double(n) * (2 + 0.375), s);
        rc = pack_text(text, n, T, s);
        if (rc) return rc;
    }
    {
        ProfScope ps(PK_KASAI, double(n) * 18, s);
        k_plcp_packed<<<gridn(n, kPlcpTile), kPlcpThreads, 0, s>>>(text, T, n, ip, isa, plcp, status);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_KASAI, double(n) * 12, s);
        k_lcp_gather<<<gridn(n, 256), 256, 0, s>>>(SA, n, plcp, lcp);
    }
    LOR_LAUNCH_CHECK();

    // Segmented overlap.
    {
        ProfScope ps(PK_OVERLAP_SCAN, double(n) * 16, s);
        const unsigned grid = unsigned(min64(cdiv(n, 256), 152 * 16));
        k_seg_argmax<<<grid, 256, 0, s>>>(SA, lcp, PK, n, bstart, starts, nseq, best);
    }
    LOR_LAUNCH_CHECK();
    const int64_t ntiles = cdiv(n, kScanTile);
    {
        ProfScope ps(PK_OVERLAP_COLLECT, double(n) * 16, s);
        rs.epoch++;
        k_seg_runs<<<unsigned(ntiles), kScanThreads, 0, s>>>(PK, bstart, lcp, best, n, run_id, d_runs,
                                                            rs.lookback, rs.tile_ctr, rs.tile_base,
                                                            rs.epoch, status);
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
        k_seg_qual<<<gridc(n), 256, 0, s>>>(SA, PK, bstart, lcp, best, n, starts, nseq, run_id, qual);
        LOR_LAUNCH_CHECK();
        rs.epoch++;
        k_seg_members<<<unsigned(ntiles), kScanThreads, 0, s>>>(SA, n, run_id, qual, mem, d_count,
                                                               rs.lookback, rs.tile_ctr, rs.tile_base,
                                                               rs.epoch, status, ntiles);
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
    }
    if (g) {
        // The member count stays on the device: everything below is sized by
        // its bound n and reads the count itself.
        uint32_t *mr, *mv;
        rc = radix_sort_pairs<uint32_t>(rs, mem, va, kb, vb, n, 0, bit_width_u64(uint64_t(n - 1)), true, &mr, &mv,
                                        false, d_count);
        if (rc) return rc;
        k_pair_count<<<gridc(n), 256, 0, s>>>(mr, n, d_count, starts, nseq, cnt);
        LOR_LAUNCH_CHECK();
        k_group_finish<<<1, 128, 0, s>>>(SA, bstart, best, cnt, starts, nseq, np, 0, g->pos_base, o.out, o.pos_off);
        LOR_LAUNCH_CHECK();
        k_group_positions<<<gridc(n), 256, 0, s>>>(mr, n, d_count, starts, nseq, 0, g->pos_base, o.pos, o.pos_cap);
        LOR_LAUNCH_CHECK();
        k_group_pos_advance<<<1, 32, 0, s>>>(g->pos_base, d_count);
        LOR_LAUNCH_CHECK();
        *h_found = 0;
        return LOR_OK;
    }
    uint32_t h_count = 0;
    LOR_CUDA_TRY(cudaMemcpyAsync(&h_count, d_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t m = h_count;
    uint32_t *mr = mem, *mv;
    if (m > 1) {
        rc = radix_sort_pairs<uint32_t>(rs, mem, va, kb, vb, m, 0, bit_width_u64(uint64_t(n - 1)), true, &mr,
                                        &mv);
        if (rc) return rc;
    }
    if (m > 0) {
        k_pair_count<<<gridc(m), 256, 0, s>>>(mr, m, nullptr, starts, nseq, cnt);
        LOR_LAUNCH_CHECK();
    }
    k_group_finish<<<1, 128, 0, s>>>(SA, bstart, best, cnt, starts, nseq, np, o.pos_base, nullptr, o.out,
                                     o.pos_off);
    LOR_LAUNCH_CHECK();
    if (m > 0 && o.pos_base < o.pos_cap) {
        k_group_positions<<<gridc(m), 256, 0, s>>>(mr, m, nullptr, starts, nseq, o.pos_base, nullptr, o.pos,
                                                   o.pos_cap);
        LOR_LAUNCH_CHECK();
    }
    *h_found = m;
    return LOR_OK;
}

}  // namespace lor

using namespace lor;

extern "C" size_t lor_batch_workspace_size(const int64_t *h_lens, int32_t npairs) {
    if (!h_lens || npairs < 1) return 0;
    int64_t nmax = 1;
    for (const Group &g : make_groups(h_lens, npairs)) nmax = g.n > nmax ? g.n : nmax;
    if (nmax > LOR_MAX_N) return 0;
    return batch_layout(nmax).total;
}

extern "C" int lor_batch_overlap(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs,
                                 lor_overlap *d_out, int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap,
                                 void *d_ws, size_t ws_bytes, lor_stream_t stream) {
    if (!h_lens || npairs < 1 || !d_out || !d_pos_off || pos_cap < 0) return LOR_ERR_INVALID_ARG;
    if (pos_cap > 0 && !d_pos) return LOR_ERR_INVALID_ARG;
    for (int i = 0; i < 2 * npairs; ++i)
        if (h_lens[i] < 0) return LOR_ERR_INVALID_ARG;
    const std::vector<Group> groups = make_groups(h_lens, npairs);
    int64_t nmax = 1, total_in = 0;
    for (const Group &g : groups) nmax = g.n > nmax ? g.n : nmax;
    for (int i = 0; i < 2 * npairs; ++i) total_in += h_lens[i];
    if (nmax > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    if (total_in > 0 && !d_ascii) return LOR_ERR_INVALID_ARG;
    const BatchLayout L = batch_layout(nmax);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    int64_t pos_base = 0;
    for (const Group &g : groups) {
        const GroupOutputs o{d_out + g.p0, d_pos_off + g.p0, d_pos, pos_cap, pos_base};
        int64_t m = 0;
        const int rc = batch_group(d_ascii ? d_ascii + g.in0 : nullptr, h_lens + 2 * g.p0, g.np, g.n, ws,
                                   ws_bytes, L, nmax, o, &m, s, nullptr);
        if (rc) return rc;
        pos_base += m;
    }
    return LOR_OK;
}

// ---------------------------------------------------------------- CUDA graph

namespace lor {
namespace {
constexpr int kGraphSaPool = 1024;   // tile counters of device-sized launches, per group
constexpr int kGraphPostPool = 64;

struct GraphExtra {
    size_t sa_pool, post_pool, pos_base, total;
};
GraphExtra graph_extra(size_t base) {
    GraphExtra E;
    E.sa_pool = align256(base);
    E.post_pool = align256(E.sa_pool + sizeof(unsigned long long) * kGraphSaPool);
    E.pos_base = align256(E.post_pool + sizeof(unsigned long long) * kGraphPostPool);
    E.total = align256(E.pos_base + sizeof(int64_t));
    return E;
}
}  // namespace
}  // namespace lor

struct lor_batch_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t *h_starts = nullptr;  // pinned: the captured copies read it at every replay
    unsigned long long kernels = 0;
};

extern "C" size_t lor_batch_graph_workspace_size(const int64_t *h_lens, int32_t npairs) {
    const size_t base = lor_batch_workspace_size(h_lens, npairs);
    return base ? graph_extra(base).total : 0;
}

extern "C" int lor_batch_graph_create(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs,
                                      lor_overlap *d_out, int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap,
                                      void *d_ws, size_t ws_bytes, lor_batch_graph **out) {
    if (!out || !h_lens || npairs < 1 || !d_out || !d_pos_off || pos_cap < 0) return LOR_ERR_INVALID_ARG;
    *out = nullptr;
    if (pos_cap > 0 && !d_pos) return LOR_ERR_INVALID_ARG;
    for (int i = 0; i < 2 * npairs; ++i)
        if (h_lens[i] < 0) return LOR_ERR_INVALID_ARG;
    const std::vector<Group> groups = make_groups(h_lens, npairs);
    int64_t nmax = 1, total_in = 0;
    for (const Group &g : groups) nmax = g.n > nmax ? g.n : nmax;
    for (int i = 0; i < 2 * npairs; ++i) total_in += h_lens[i];
    if (nmax > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    if (total_in > 0 && !d_ascii) return LOR_ERR_INVALID_ARG;
    const BatchLayout L = batch_layout(nmax);
    const GraphExtra E = graph_extra(L.total);
    if (!d_ws || ws_bytes < E.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    char *ws = (char *)d_ws;

    lor_batch_graph *G = new lor_batch_graph();
    size_t nst = 0;
    for (const Group &g : groups) nst += size_t(2 * g.np + 1);
    if (cudaMallocHost(&G->h_starts, sizeof(int32_t) * nst) != cudaSuccess) {
        delete G;
        return LOR_ERR_CUDA;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFreeHost(G->h_starts);
        delete G;
        return LOR_ERR_CUDA;
    }
    int rc = LOR_OK;
    capture_begin();
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = LOR_ERR_CUDA;
    if (rc == LOR_OK) {
        int64_t *pos_base = (int64_t *)(ws + E.pos_base);
        if (cudaMemsetAsync(pos_base, 0, sizeof(int64_t), cs) != cudaSuccess) rc = LOR_ERR_CUDA;
        size_t st = 0;
        for (size_t gi = 0; gi < groups.size() && rc == LOR_OK; ++gi) {
            const Group &g = groups[gi];
            GroupGraph gg;
            gg.sa_pool = (unsigned long long *)(ws + E.sa_pool);
            gg.sa_pool_size = kGraphSaPool;
            gg.post_pool = (unsigned long long *)(ws + E.post_pool);
            gg.post_pool_size = kGraphPostPool;
            gg.pos_base = pos_base;
            gg.h_starts = G->h_starts + st;
            st += size_t(2 * g.np + 1);
            const GroupOutputs o{d_out + g.p0, d_pos_off + g.p0, d_pos, pos_cap, 0};
            int64_t found = 0;
            rc = batch_group(d_ascii ? d_ascii + g.in0 : nullptr, h_lens + 2 * g.p0, g.np, g.n, ws, L.total, L,
                             nmax, o, &found, cs, &gg);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (rc == LOR_OK && (e != cudaSuccess || !graph)) rc = LOR_ERR_CUDA;
        G->graph = graph;
    }
    G->kernels = capture_end();
    cudaStreamDestroy(cs);
    if (rc == LOR_OK && cudaGraphInstantiate(&G->exec, G->graph, 0) != cudaSuccess) rc = LOR_ERR_CUDA;
    if (rc != LOR_OK) {
        cudaGetLastError();
        lor_batch_graph_destroy(G);
        return rc;
    }
    *out = G;
    return LOR_OK;
}

extern "C" int lor_batch_graph_launch(lor_batch_graph *g, lor_stream_t stream) {
    if (!g || !g->exec) return LOR_ERR_INVALID_ARG;
    if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) return LOR_ERR_CUDA;
    note_graph_launches(g->kernels);
    return LOR_OK;
}

extern "C" int64_t lor_batch_graph_kernels(const lor_batch_graph *g) { return g ? int64_t(g->kernels) : 0; }

extern "C" int lor_batch_graph_destroy(lor_batch_graph *g) {
    if (!g) return LOR_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->h_starts) cudaFreeHost(g->h_starts);
    delete g;
    return LOR_OK;
}
