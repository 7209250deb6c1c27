// dc3.cu -- suffix array by DC3 / skew (Section 3, Steps 1-3; Tables 1-3).
//
// One recursion level on a string s[0..n) over codes [1..K] (0 = padding):
//   Step 1  sample positions C = {i : i mod 3 != 0} (plus the dummy position
//           n when n mod 3 == 1) get keys from the symbols starting at i
//           (the triple [t_i t_i+1 t_i+2]; level 0 may use a longer prefix),
//           are radix sorted and named; R = R1 (i mod 3 == 1) followed by R2
//           (i mod 3 == 2) holds the names.  Non-unique names -> recurse on R.
//           The suffix array of R gives rank(S_i) for every sample i.
//   Step 2  nonsample positions (i mod 3 == 0) ordered by (t_i, rank(S_i+1)):
//           take them in the order of rank(S_i+1) from the sample order, then
//           one stable radix sort by t_i.
//   Step 3  merge: sample i in B1 against nonsample j compares
//           (t_i, rank(S_i+1)) with (t_j, rank(S_j+1)); i in B2 compares
//           (t_i, t_i+1, rank(S_i+2)) with (t_j, t_j+1, rank(S_j+2)).  (The
//           paper prints rank(S_i+1) for B2; i+2 is the sample position.)
// The host drives the recursion and reads one count per level.
#include <atomic>
#include <cstdlib>
#include <vector>

#include "batch.cuh"
#include "dc3_packed.cuh"
#include "radix.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_dc3)

namespace lor {
namespace {

struct LevelSizes {
    int64_t n, n0, n1, n2, n02;
};
inline LevelSizes level_sizes(int64_t n) {
    LevelSizes z;
    z.n = n;
    z.n0 = (n + 2) / 3;
    z.n1 = (n + 1) / 3;
    z.n2 = n / 3;
    z.n02 = z.n0 + z.n2;
    return z;
}

// Lengths of every level the recursion could reach.
std::vector<int64_t> level_chain(int64_t n) {
    std::vector<int64_t> c{n};
    while (c.back() > 3 && c.size() < 96) c.push_back(level_sizes(c.back()).n02);
    return c;
}

constexpr size_t kPad = 4;  // zero symbols kept after every reduced string

// Tiles of the level-0 nonsample split (entries of SAR per tile, 16 per
// thread) and the number of tile ranges its scan works in.
constexpr int kSpItems = 8;
constexpr int kSpTile = 256 * kSpItems;
constexpr int kSpRanges = 512;

struct Dc3Layout {
    size_t ns_table = 0;  // the split's per-tile starts (level 0)
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t tbl = 0;
    int64_t tbl_entries = 0;
    size_t split = 0;  // merge-path partition of the largest level
    size_t t64[3] = {0, 0, 0};
    size_t t32[6] = {0, 0, 0, 0, 0, 0};
    int64_t max_m = 0;
    std::vector<int64_t> lev_n;
    std::vector<size_t> lev_R, lev_SAR, lev_NS;
    size_t total = 0;
};

// Entries of the dense naming table: enough for 24-bit keys at scale, and
// never much larger than the sample.
int64_t dense_entries(int64_t max_m) {
    int64_t e = int64_t(1) << 16;
    while (e < (int64_t(1) << 24) && e < 4 * max_m) e <<= 1;
    return e;
}

Dc3Layout dc3_layout(int64_t n) {
    Dc3Layout L;
    L.lev_n = level_chain(n);
    L.max_m = level_sizes(n).n02;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(L.max_m);
    L.lookback = take(L.lookback_bytes);
    L.tbl_entries = dense_entries(L.max_m);
    L.tbl = take(sizeof(uint32_t) * size_t(L.tbl_entries));
    // t64[1], t64[2] are adjacent: together they hold the merge records.
    for (int i = 0; i < 3; ++i) L.t64[i] = take(sizeof(uint64_t) * size_t(L.max_m));
    L.split = take(sizeof(int64_t) * size_t(cdiv(n, 1024) + 2));
    for (int i = 0; i < 6; ++i) L.t32[i] = take(sizeof(uint32_t) * size_t(L.max_m));
    L.ns_table = take(sizeof(uint32_t) * 256 * size_t(cdiv(L.max_m, kSpTile) + kSpRanges));
    for (size_t l = 0; l < L.lev_n.size(); ++l) {
        const int64_t m = level_sizes(L.lev_n[l]).n02;
        L.lev_R.push_back(take(sizeof(int32_t) * (size_t(m) + kPad)));
        L.lev_SAR.push_back(take(sizeof(int32_t) * size_t(m)));
        L.lev_NS.push_back(take(sizeof(int32_t) * size_t(m)));
    }
    L.total = off;
    return L;
}

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ int64_t sample_pos(int64_t j, int64_t n0) {
    return j < n0 ? 3 * j + 1 : 3 * (j - n0) + 2;
}

// Step 1 keys: kchars symbols starting at the sample position, `bits` bits
// each, most significant first; positions >= n read as 0.  At level 0 the
// text codes are validated (must lie in [1, maxc]) and clamped.
template <typename CharT, typename KeyT, bool kValidate>
__global__ void __launch_bounds__(256) k_sample_keys(const CharT *__restrict__ s, int64_t n,
                                                     int64_t n0, int64_t n02, int first, int kchars,
                                                     uint64_t radix, int64_t maxc, KeyT *__restrict__ keys,
                                                     int *status) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n02) return;
    const int64_t p = sample_pos(j, n0);
    KeyT key = 0;
    bool bad = false;
    for (int t = first; t < kchars; ++t) {
        const int64_t q = p + t;
        int64_t c = q < n ? int64_t(s[q]) : 0;
        if (kValidate && q < n && (c < 1 || c > maxc)) {
            bad = true;
            c = c < 1 ? 1 : maxc;
        }
        key = key * KeyT(radix) + KeyT(c);
    }
    if (kValidate && j == 0 && n > 0) {
        const int64_t c = int64_t(s[0]);
        if (c < 1 || c > maxc) bad = true;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
    keys[j] = key;
}

// Level-0 keys staged through shared memory.  Block (x, c) makes the keys of
// kKeyTile consecutive samples of one class: c = 0 positions 3j+1 (j < n0,
// stored at j), c = 1 positions 3j+2 (j < n2, stored at n0 + j).  The text
// bytes the tile needs are read once, coalesced, and validated (codes must
// lie in [1, maxc]); every radix pass's digit histogram is counted on the
// way, so the sort needs no separate histogram read of the keys.
constexpr int kKeyTile = 4096;
constexpr int kKeyMaxChars = 64;

// The key is formed by Horner's rule over 32-bit chunks of `chunk` symbols
// (radix^chunk <= 2^32), the chunks joined with one 64-bit multiply-add each.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_sample_keys0(const uint8_t *__restrict__ s, int64_t n, int64_t n0,
                                                      int64_t n2, int kchars, int chunk, uint32_t radix,
                                                      int64_t maxc, KeyT *__restrict__ keys, int npasses,
                                                      int end_bit, int dbits, uint32_t *__restrict__ hist,
                                                      int *status) {
    __shared__ uint8_t txt[3 * kKeyTile + kKeyMaxChars];
    __shared__ uint32_t sh[kMaxPasses * kRadix];
    const int tid = threadIdx.x;
    const int cls = int(blockIdx.y);
    const int64_t ncls = cls == 0 ? n0 : n2;
    const int64_t j0 = int64_t(blockIdx.x) * kKeyTile;
    if (j0 >= ncls) return;  // uniform over the block
    const int nj = int(min64(int64_t(kKeyTile), ncls - j0));
    const int64_t p0 = 3 * j0 + 1 + cls;
    const int span = 3 * (nj - 1) + kchars;
    bool bad = false;
    for (int i = tid; i < span; i += 256) {
        const int64_t q = p0 + i;
        uint32_t c = 0;
        if (q < n) {
            c = s[q];
            if (c < 1 || c > uint32_t(maxc)) {  // keeps the key inside its range
                bad = true;
                c = c < 1 ? 1u : uint32_t(maxc);
            }
        }
        txt[i] = uint8_t(c);
    }
    for (int i = tid; i < npasses * kRadix; i += 256) sh[i] = 0;
    if (blockIdx.x == 0 && cls == 0 && tid == 0 && n > 0) {
        const uint32_t c = s[0];
        if (c < 1 || c > uint32_t(maxc)) bad = true;
    }
    __syncthreads();
    KeyT *out = keys + (cls == 0 ? 0 : n0) + j0;
    const int tail = kchars % chunk;
    uint64_t pw_chunk = 1, pw_tail = 1;
    for (int t = 0; t < chunk; ++t) pw_chunk *= radix;
    for (int t = 0; t < tail; ++t) pw_tail *= radix;
    for (int k = tid; k < nj; k += 256) {
        const uint8_t *w = txt + 3 * k;
        uint64_t key = 0;
        int t = 0;
        for (; t + chunk <= kchars; t += chunk) {
            uint32_t part = 0;
            for (int u = 0; u < chunk; ++u) part = part * radix + w[t + u];
            key = key * pw_chunk + part;
        }
        if (tail) {
            uint32_t part = 0;
            for (int u = 0; u < tail; ++u) part = part * radix + w[t + u];
            key = key * pw_tail + part;
        }
        out[k] = KeyT(key);
        if (hist)
            for (int p = 0; p < npasses; ++p) {
                const int sft = p * dbits;
                atomicAdd(&sh[p * kRadix + digit_of(key, sft, digit_mask(sft, end_bit, dbits))], 1u);
            }
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
    if (hist) {
        __syncthreads();
        for (int i = tid; i < npasses * kRadix; i += 256)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

// Step 1 naming: name(j) = 1 + number of key changes in sorted[0..j].
// Writes R[val] = name, SA_R[j] = val, and the name count.  Persistent: a
// resident grid claims tiles until it draws one past the end (launched by
// LOR_PTILE_LAUNCH).
template <typename KeyT>
__global__ void __launch_bounds__(kScanThreads) k_name(const KeyT *__restrict__ keys,
                                                       const uint32_t *__restrict__ vals, int64_t m,
                                                       int32_t *__restrict__ R, int32_t *__restrict__ SAR,
                                                       int32_t *__restrict__ NS, uint32_t *n_names, uint64_t *lb,
                                                       unsigned long long *ctr,
                                                       unsigned long long tile_base, uint32_t epoch,
                                                       int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    const int64_t ntiles = cdiv(m > 0 ? m : 1, kScanTile);
    for (;;) {
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) break;  // uniform over the block
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    KeyT prev = (base > 0 && base - 1 < m) ? keys[base - 1] : KeyT(0);
    KeyT kk[kScanItems];
    load_run<KeyT, kScanItems>(keys, base, m, KeyT(0), kk);
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < m) {
            const uint32_t f = (j == 0 || kk[i] != prev) ? 1u : 0u;
            flags |= f << i;
            cnt += f;
            prev = kk[i];
        }
    }
    uint32_t vv[kScanItems];
    load_run<uint32_t, kScanItems>(vals, base, m, 0u, vv);
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) s_prefix = p;
    }
    __syncthreads();
    uint32_t name = s_prefix + excl;
    int32_t nm[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        name += (flags >> i) & 1u;
        nm[i] = int32_t(name);
        const int64_t j = base + i;
        if (j < m) {
            if (R) R[vv[i]] = int32_t(name);
            if (j == m - 1) *n_names = name;
        }
    }
    store_run<int32_t, kScanItems>(SAR, base, m, reinterpret_cast<const int32_t(&)[kScanItems]>(vv));
    store_run<int32_t, kScanItems>(NS, base, m, nm);
    __syncthreads();  // s_tile and s_prefix are reused by the next tile
    }
}

// Naming after a two-stage sort: equality of triples is checked on the
// string itself (the last sort key holds only the first symbol).
template <typename CharT>
__global__ void __launch_bounds__(kScanThreads) k_name_gather(
    const uint32_t *__restrict__ vals, int64_t m, const CharT *__restrict__ s, int64_t n,
    int64_t n0, int32_t *__restrict__ R, int32_t *__restrict__ SAR, int32_t *__restrict__ NS,
    uint32_t *n_names, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base,
    uint32_t epoch, int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    auto ch = [&](int64_t q) -> int64_t { return q < n ? int64_t(s[q]) : 0; };
    int64_t pp = (base > 0 && base - 1 < m) ? sample_pos(vals[base - 1], n0) : -1;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < m) {
            const int64_t p = sample_pos(vals[j], n0);
            const bool same = j > 0 && ch(p) == ch(pp) && ch(p + 1) == ch(pp + 1) &&
                              ch(p + 2) == ch(pp + 2);
            const uint32_t f = same ? 0u : 1u;
            flags |= f << i;
            cnt += f;
            pp = p;
        }
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) s_prefix = p;
    }
    __syncthreads();
    uint32_t name = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < m) {
            name += (flags >> i) & 1u;
            const uint32_t v = vals[j];
            if (R) R[v] = int32_t(name);
            SAR[j] = int32_t(v);
            NS[j] = int32_t(name);
            if (j == m - 1) *n_names = name;
        }
    }
}

// First symbol of each sample in sorted order (second stage of a wide sort).
template <typename CharT>
__global__ void k_first_char(const uint32_t *__restrict__ vals, int64_t m, const CharT *__restrict__ s,
                             int64_t n, int64_t n0, uint32_t *__restrict__ keys) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t p = sample_pos(vals[j], n0);
    keys[j] = p < n ? uint32_t(s[p]) : 0u;
}

// rank(S_i) for every sample after recursion: rankR[SA_R[j]] = j + 1.
__global__ void k_rank_scatter(const int32_t *__restrict__ SAR, int64_t m, int32_t *__restrict__ rankR,
                               int *status) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t r = SAR[j];
    if (r < 0 || r >= m) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    rankR[r] = int32_t(j + 1);
}

// Step 2 gather: nonsample positions 3r for every B1 sample r in rank order,
// keyed by their first symbol (order-preserving compaction by look-back).
// The value emitted is the group index r (the nonsample position is 3r).
template <typename CharT>
__global__ void __launch_bounds__(kScanThreads) k_nonsample(
    const int32_t *__restrict__ SAR, int64_t m, int64_t n0, const CharT *__restrict__ s, int64_t n,
    uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, uint64_t *lb, unsigned long long *ctr,
    unsigned long long tile_base, uint32_t epoch, int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    int32_t r[kScanItems];
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        r[i] = j < m ? SAR[j] : -1;
        if (r[i] >= 0 && r[i] < n0) cnt++;
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) s_prefix = p;
    }
    __syncthreads();
    uint32_t o = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (r[i] >= 0 && r[i] < n0) {
            const int64_t q = 3 * int64_t(r[i]);
            keys[o] = q < n ? uint32_t(s[q]) : 0u;
            vals[o] = uint32_t(r[i]);
            ++o;
        }
    }
}

// ---- Step 3: merge of sample and nonsample suffixes (merge path)
//
// Every comparison of Step 3 reads two symbols and one or two ranks next to a
// position.  For the group of positions 3t, 3t+1, 3t+2 all of them sit in one
// record: symbols t_3t..t_3t+3 and rank(S_3t+1), rank(S_3t+2), rank(S_3t+4).
// The records are written by a streaming pass over t, so a merged suffix
// costs a single gather of its group's record.

template <typename CharT>
struct GroupRec;
template <>
struct __align__(16) GroupRec<uint8_t> {
    uint32_t c4;  // four symbols, byte k = t_3t+k
    int32_t r1, r2, r4;
};
template <>
struct __align__(32) GroupRec<int32_t> {
    int32_t c[4];
    int32_t r1, r2, r4, pad;
};
__device__ __forceinline__ int32_t rec_ch(const GroupRec<uint8_t> &g, int k) {
    return int32_t((g.c4 >> (8 * k)) & 0xFFu);
}
__device__ __forceinline__ int32_t rec_ch(const GroupRec<int32_t> &g, int k) { return g.c[k]; }

// Record of group t: rank(S_x) is rankR[(x-1)/3] for x = 1 mod 3 (the dummy
// x = n included), rankR[n0 + (x-2)/3] for x = 2 mod 3, and 0 past the end.
template <typename CharT>
__global__ void k_group_records(const CharT *__restrict__ s, int64_t n, int64_t n0, int64_t n2,
                                const int32_t *__restrict__ rankR, GroupRec<CharT> *__restrict__ rec) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n0) return;
    const int64_t q = 3 * t;
    GroupRec<CharT> g;
    int32_t c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = q + k < n ? int32_t(s[q + k]) : 0;
    if constexpr (sizeof(CharT) == 1) {
        g.c4 = uint32_t(c[0]) | (uint32_t(c[1]) << 8) | (uint32_t(c[2]) << 16) | (uint32_t(c[3]) << 24);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) g.c[k] = c[k];
        g.pad = 0;
    }
    g.r1 = rankR[t];
    g.r2 = t < n2 ? rankR[n0 + t] : 0;
    g.r4 = t + 1 < n0 ? rankR[t + 1] : 0;
    rec[t] = g;
}

// Nonsample suffix 3t with its comparison key, in nonsample order (written
// by k_nonsample_split at level 0): t, t_3t | t_3t+1 << 8, rank(S_3t+1),
// rank(S_3t+2).
struct __align__(16) BRec16 {
    int32_t t;
    uint32_t c01;
    int32_t r1, r2;
};

template <typename CharT>
struct MergeIn {
    const GroupRec<CharT> *rec;
    int32_t n0;
    const int32_t *A;  // sample order (reduced-string indices), dummy skipped
    int64_t na;
    const uint32_t *B;  // nonsample order (group indices t; position 3t)
    int64_t nb;
    const BRec16 *Bx;  // when set: the nonsample records in order (B unused)
    const uint64_t *Ax;  // when set: the sample keys in sample order, aligned with A (no record gathers)
};

// Sample suffix p: key (t_p, rank(S_p+1)) for p = 1 mod 3 (marked c1 = -1),
// (t_p, t_p+1, rank(S_p+2)) for p = 2 mod 3.
struct ARec { int32_t pos, c0, c1, r; };
// Nonsample suffix q: t_q, t_q+1, rank(S_q+1), rank(S_q+2).
struct BRec { int32_t pos, c0, c1, r1, r2; };

__device__ __forceinline__ int32_t a_group(int32_t r, int32_t n0) { return r < n0 ? r : r - n0; }

template <typename CharT>
__device__ __forceinline__ ARec make_a(const GroupRec<CharT> &g, int32_t r, int32_t n0) {
    ARec x;
    if (r < n0) {
        x.pos = 3 * r + 1;
        x.c0 = rec_ch(g, 1);
        x.c1 = -1;
        x.r = g.r2;
    } else {
        x.pos = 3 * (r - n0) + 2;
        x.c0 = rec_ch(g, 2);
        x.c1 = rec_ch(g, 3);
        x.r = g.r4;
    }
    return x;
}
// A sample's comparison key packed in 8 bytes (level 0, written by the
// bucketed scatter of SampleKeySrc): rank in the low word, then t_p and, for
// p = 2 mod 3, t_p+1 (for p = 1 mod 3 that byte holds t_p-1, which the
// comparison does not read; the class comes from the reduced-string index).
__device__ __forceinline__ ARec unpack_a(uint64_t w, int32_t r, int32_t n0) {
    ARec x;
    x.pos = r < n0 ? 3 * r + 1 : 3 * (r - n0) + 2;
    x.r = int32_t(uint32_t(w));
    x.c0 = int32_t((w >> 32) & 0xFFu);
    x.c1 = r < n0 ? -1 : int32_t((w >> 40) & 0xFFu);
    return x;
}

template <typename CharT>
__device__ __forceinline__ BRec make_b(const GroupRec<CharT> &g, uint32_t t) {
    BRec y;
    y.pos = int32_t(3 * t);
    y.c0 = rec_ch(g, 0);
    y.c1 = rec_ch(g, 1);
    y.r1 = g.r1;
    y.r2 = g.r2;
    return y;
}
__device__ __forceinline__ BRec make_bx(const BRec16 &g) {
    BRec y;
    y.pos = 3 * g.t;
    y.c0 = int32_t(g.c01 & 0xFFu);
    y.c1 = int32_t((g.c01 >> 8) & 0xFFu);
    y.r1 = g.r1;
    y.r2 = g.r2;
    return y;
}
// Is the sample suffix x smaller than the nonsample suffix y?
__device__ __forceinline__ bool a_less_b(const ARec &x, const BRec &y) {
    if (x.c0 != y.c0) return x.c0 < y.c0;
    if (x.c1 < 0) return x.r < y.r1;
    if (x.c1 != y.c1) return x.c1 < y.c1;
    return x.r < y.r2;
}

// A merge tile is 1024 outputs: 512 threads x 2, 256 x 4 or 128 x 8
// (tune_config().merge_items).  Wide blocks with few items each keep the most
// record gathers in flight; with the level-0 records carried in order there is
// nothing to gather and more items per thread amortise the merge-path search.
constexpr int kMergeTile = 1024;
static_assert(kMergeTile >= 1024, "the workspace holds a partition entry per 1024 merged suffixes");

// Number of sample suffixes among the first d merged suffixes.
template <typename CharT>
__device__ int64_t merge_split(const MergeIn<CharT> &a, int64_t d) {
    int64_t lo = d - a.nb > 0 ? d - a.nb : 0;
    int64_t hi = d < a.na ? d : a.na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t r = a.A[mid];
        const ARec x = a.Ax ? unpack_a(a.Ax[mid], r, a.n0) : make_a(a.rec[a_group(r, a.n0)], r, a.n0);
        BRec y;
        if (a.Bx) {
            y = make_bx(a.Bx[d - 1 - mid]);
        } else {
            const uint32_t t = a.B[d - 1 - mid];
            y = make_b(a.rec[t], t);
        }
        if (a_less_b(x, y)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename CharT>
__global__ void k_merge_partition(MergeIn<CharT> a, int64_t ntiles, int64_t *__restrict__ split) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    const int64_t tot = a.na + a.nb;
    const int64_t d = t * kMergeTile < tot ? t * kMergeTile : tot;
    split[t] = merge_split(a, d);
}

template <typename CharT, int kMergeItems>
__global__ void __launch_bounds__(kMergeTile / kMergeItems) k_merge(MergeIn<CharT> a,
                                                                    const int64_t *__restrict__ split,
                                                                    int32_t *__restrict__ out, int *status) {
    constexpr int kMergeThreads = kMergeTile / kMergeItems;
    __shared__ ARec As[kMergeTile];
    __shared__ BRec Bs[kMergeTile];
    __shared__ int32_t Os[kMergeTile];
    const int64_t t = blockIdx.x;
    const int64_t tot = a.na + a.nb;
    const int64_t d0 = t * kMergeTile;
    const int64_t d1 = d0 + kMergeTile < tot ? d0 + kMergeTile : tot;
    // Valid inputs give monotone splits; the clamps keep every access in
    // bounds (and report it) if the inputs were not suffix-consistent.
    int64_t a0 = split[t], a1 = split[t + 1];
    const int64_t a0c = min64(max64(a0, max64(0, d0 - a.nb)), min64(d0, a.na));
    int64_t a1c = min64(max64(a1, max64(0, d1 - a.nb)), min64(d1, a.na));
    a1c = min64(max64(a1c, a0c), a0c + (d1 - d0));
    if ((a0c != a0 || a1c != a1) && threadIdx.x == 0) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
    a0 = a0c;
    a1 = a1c;
    const int64_t b0 = d0 - a0, b1 = d1 - a1;
    const int na = int(a1 - a0), nb = int(b1 - b0), nt = int(d1 - d0);
    // Load the tile: all indices first, then all record gathers, so that each
    // thread keeps kMergeItems independent loads in flight.
    if (a.Bx && a.Ax) {
        // Both orders arrive with their keys: no gathers at all.
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            if (sl < na) As[sl] = unpack_a(a.Ax[a0 + sl], a.A[a0 + sl], a.n0);
            else if (sl < nt) Bs[sl - na] = make_bx(a.Bx[b0 + sl - na]);
        }
    } else if (a.Bx) {
        // Nonsample records arrive in order: only the samples are gathered.
        int32_t idx[kMergeItems];
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            idx[k] = sl < na ? a.A[a0 + sl] : 0;
        }
        GroupRec<CharT> g[kMergeItems];
        BRec16 bx[kMergeItems];
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            if (sl < na) g[k] = a.rec[a_group(idx[k], a.n0)];
            else if (sl < nt) bx[k] = a.Bx[b0 + sl - na];
        }
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            if (sl < na) As[sl] = make_a(g[k], idx[k], a.n0);
            else if (sl < nt) Bs[sl - na] = make_bx(bx[k]);
        }
    } else {
        int32_t idx[kMergeItems];
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            idx[k] = sl < na ? a.A[a0 + sl] : (sl < nt ? int32_t(a.B[b0 + sl - na]) : 0);
        }
        GroupRec<CharT> g[kMergeItems];
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            if (sl < nt) g[k] = a.rec[sl < na ? a_group(idx[k], a.n0) : idx[k]];
        }
#pragma unroll
        for (int k = 0; k < kMergeItems; ++k) {
            const int sl = int(threadIdx.x) + k * kMergeThreads;
            if (sl < na) As[sl] = make_a(g[k], idx[k], a.n0);
            else if (sl < nt) Bs[sl - na] = make_b(g[k], uint32_t(idx[k]));
        }
    }
    __syncthreads();
    const int dl = min(int(threadIdx.x) * kMergeItems, nt);
    int lo = max(0, dl - nb), hi = min(dl, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a_less_b(As[mid], Bs[dl - 1 - mid])) lo = mid + 1;
        else hi = mid;
    }
    int ia = lo, ib = dl - lo;
#pragma unroll
    for (int k = 0; k < kMergeItems; ++k) {
        const int o = dl + k;
        if (o >= nt) break;
        const bool take_a = ib >= nb || (ia < na && a_less_b(As[ia], Bs[ib]));
        Os[o] = take_a ? As[ia++].pos : Bs[ib++].pos;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += kMergeThreads) out[d0 + i] = Os[i];
}

// ---- Step 2 at level 0 with the records: the nonsample suffixes 3t in the
// order of rank(S_3t+1) (that is, of the B1 samples in SAR) are split stably
// by their first symbol t_3t, and each carries its record (gathered here once,
// from the group records) so that the merge reads them in order.

// hist[c] = number of nonsample positions 3t (t < n0) holding symbol c.
__global__ void k_first_sym_hist(const uint8_t *__restrict__ s, int64_t n0, uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[kRadix];
    sh[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n0; t += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&sh[s[3 * t]], 1u);
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

constexpr int kNsItems = 8;
constexpr int kNsTile = kSortThreads * kNsItems;

struct NsSmem {
    BRec16 rec[kNsTile];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t local_start[kRadix];
    long long gbase[kRadix];
    uint32_t scratch[kSortWarps + 1];
    uint32_t count;
    long long tile;
};

// Marks a B1 sample's merge key (bit 63 of the packed key; no reader of the
// key's comparison bytes looks at it).
constexpr uint64_t kB1Flag = uint64_t(1) << 63;

// Every sample's merge key (Step 3), made in reduced-string order x from the
// text and the ranks (all read in sequence) and keyed by the sample's index
// in sample order, j = rank(S_x) - 1, for a bucketed scatter into Ax[j]:
//   B1 sample p = 3x+1: rank(S_p+1) in the low word, t_p in byte 4 and t_p-1
//       (the first symbol of the nonsample 3x) in byte 5;
//   B2 sample p = 3x'+2 (x = n0 + x'): rank(S_p+2), t_p, t_p+1.
// (x = n0 - 1 is the dummy sample at p = n when n mod 3 == 1: symbols 0.)
struct SampleKeySrc {
    const uint8_t *s;
    const int32_t *Rl;
    int64_t n, n0, n2;
    __device__ __forceinline__ void load(int64_t x, bool valid, uint32_t &k, uint64_t &v) const {
        if (!valid) {
            k = 0;
            v = 0;
            return;
        }
        k = uint32_t(Rl[x] - 1);
        if (x < n0) {
            const int64_t p = 3 * x + 1;
            const uint64_t c0 = p < n ? s[p] : 0, cm = s[p - 1];
            const uint32_t r = x < n2 ? uint32_t(Rl[n0 + x]) : 0u;
            v = uint64_t(r) | (c0 << 32) | (cm << 40) | kB1Flag;
        } else {
            const int64_t xp = x - n0, p = 3 * xp + 2;
            const uint64_t c0 = p < n ? s[p] : 0, c1 = p + 1 < n ? s[p + 1] : 0;
            const uint32_t r = xp + 1 < n0 ? uint32_t(Rl[xp + 1]) : 0u;
            v = uint64_t(r) | (c0 << 32) | (c1 << 40);
        }
    }
    // asks the L2 for the ranks and text that samples [b, b + c) read
    __device__ __forceinline__ void prefetch(int64_t b, int64_t c) const {
        const int64_t e = b + c;
        if (b < n0) {
            const int64_t e1 = e < n0 ? e : n0;
            prefetch_inside(Rl + b, Rl + e1);
            if (b < n2) prefetch_inside(Rl + n0 + b, Rl + n0 + (e1 < n2 ? e1 : n2));
            prefetch_inside(s + 3 * b, s + (3 * e1 < n ? 3 * e1 : n));
        }
        if (e > n0) {
            const int64_t b2 = (b > n0 ? b : n0) - n0, e2 = e - n0;
            prefetch_inside(Rl + b, Rl + e);
            prefetch_inside(Rl + b2 + 1, Rl + (e2 + 1 < n0 ? e2 + 1 : n0));
            prefetch_inside(s + 3 * b2 + 2, s + (3 * e2 + 2 < n ? 3 * e2 + 2 : n));
        }
    }
};

// Ax[j] = v for the (j, v) pairs of the bucketed scatter above (j distinct).
__global__ void k_scatter_u64(const uint32_t *__restrict__ key, const uint64_t *__restrict__ val, int64_t m,
                              uint64_t *__restrict__ dst, int64_t bound, int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t j = key[i];
    if (int64_t(j) >= bound) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    dst[j] = val[i];
}

// Step 2 at level 0: the nonsample suffixes 3x in the order of
// rank(S_3x+1) -- the B1 samples x in sample order SAR -- split stably by
// their first symbol t_3x, each with its merge record (t, t_3x | t_3x+1 << 8,
// rank(S_3x+1) = j + 1, rank(S_3x+2)), all read in sequence from SAR and Ax.
// Three steps with no inter-block wait: per tile of SAR, the number of B1
// samples per first symbol; the tiles' starts per symbol (an exclusive scan
// over the tiles, from the symbols' starts); per tile, each record written at
// its tile's start plus its stable rank inside the tile.

// The split's kernels read SAR and the keys tile by tile, the next tile of a
// block's stride prefetched into shared memory by bulk copies.
// (dynamic shared memory: more than the 48 KB a static allocation may take)
using NsTiles = BulkPair<int32_t, uint64_t, kSpTile>;
struct NsCountSmem {
    BulkOne<uint64_t, kSpTile> T;  // the count reads the keys only (they carry the B1 flag and t_3x)
    uint32_t h[kRadix];
};
struct NsWriteSmem {
    NsTiles T;
    uint32_t wh[kSortWarps][kRadix];
};

// kSymBits: bits of the symbols ranked (4 when every code is below 16, as
// for DNA: four ballots find a lane's peers instead of nine).
template <int kSymBits>
__global__ void __launch_bounds__(kSortThreads) k_ns_count(const uint64_t *__restrict__ Ax, int64_t n02,
                                                          uint32_t *__restrict__ cnt, int *status) {
    constexpr uint32_t kNone = 1u << kSymBits, kMask = kNone - 1u;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    NsCountSmem &S = *reinterpret_cast<NsCountSmem *>(smem_raw);
    BulkOne<uint64_t, kSpTile> &T = S.T;
    uint32_t *h = S.h;
    const int tid = threadIdx.x;
    const int64_t ntiles = cdiv(n02, kSpTile);
    const uint64_t limit = wait_limit_ns();
    BulkOneLoader<uint64_t, kSpTile> ld(T, Ax, n02);
    int64_t tile = blockIdx.x;
    if (tid == 0) ld.issue(tile, 0);
    for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const int64_t nxt = tile + gridDim.x;
        if (tid == 0 && nxt < ntiles) ld.issue(nxt, b ^ 1);
        h[tid] = 0;
        const bool whole = ld.whole(tile);
        const bool ok = ld.wait(tile, b, limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, 0, LOR_ERR_TIMEOUT);
                ld.drain(tile, b, nxt, limit);
            }
            __syncthreads();
            return;
        }
        uint32_t d[kSpItems];
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) {
            const int loc = i * kSortThreads + tid;
            const int64_t idx = tile * kSpTile + loc;
            uint64_t w = 0;
            if (whole) w = T.a[b][loc];
            else if (idx < n02) w = Ax[idx];
            d[i] = (w & kB1Flag) ? uint32_t(w >> 40) & kMask : kNone;
        }
        // one shared-memory add per distinct symbol of a warp (few symbols:
        // per-lane adds would all queue on the same words)
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) {
            const uint32_t peers = warp_peers_bits<kSymBits + 1>(d[i]);
            if (d[i] < kNone && __popc(peers & lanemask_lt()) == 0) atomicAdd(&h[d[i]], uint32_t(__popc(peers)));
        }
        __syncthreads();
        cnt[tile * kRadix + tid] = h[tid];
        __syncthreads();  // the counts and the buffer are reused
    }
}

// Per digit (thread), the sum of the counts of each range of tiles.
__global__ void __launch_bounds__(kRadix) k_ns_scan_ranges(const uint32_t *__restrict__ cnt, int64_t ntiles,
                                                          int64_t per, uint32_t *__restrict__ part) {
    const int d = threadIdx.x;
    const int64_t t0 = blockIdx.x * per, t1 = min64(t0 + per, ntiles);
    uint32_t sum = 0;
    for (int64_t t = t0; t < t1; ++t) sum += cnt[t * kRadix + d];
    part[blockIdx.x * kRadix + d] = sum;
}

// Per digit, the ranges' starts: the digit's start plus the counts before.
__global__ void __launch_bounds__(kRadix) k_ns_scan_starts(uint32_t *__restrict__ part, int nranges,
                                                          const uint32_t *__restrict__ offsets) {
    const int d = threadIdx.x;
    uint32_t run = offsets[d];
    for (int r = 0; r < nranges; ++r) {
        const uint32_t v = part[r * kRadix + d];
        part[r * kRadix + d] = run;
        run += v;
    }
}

// Per digit, every tile's start (in place of its count).
__global__ void __launch_bounds__(kRadix) k_ns_scan_tiles(uint32_t *__restrict__ cnt, int64_t ntiles, int64_t per,
                                                         const uint32_t *__restrict__ part) {
    const int d = threadIdx.x;
    const int64_t t0 = blockIdx.x * per, t1 = min64(t0 + per, ntiles);
    uint32_t run = part[blockIdx.x * kRadix + d];
    for (int64_t t = t0; t < t1; ++t) {
        const uint32_t v = cnt[t * kRadix + d];
        cnt[t * kRadix + d] = run;
        run += v;
    }
}

// Every record at its tile's start for its first symbol plus its stable rank
// in the tile (each warp owns a run of 512 consecutive entries: items in
// order, lanes in order).
template <int kSymBits>
__global__ void __launch_bounds__(kSortThreads, 3) k_ns_write(const int32_t *__restrict__ SAR,
                                                             const uint64_t *__restrict__ Ax, int64_t n02, int64_t n0,
                                                             const uint32_t *__restrict__ start,
                                                             BRec16 *__restrict__ out, int *status) {
    constexpr uint32_t kNone = 1u << kSymBits, kMask = kNone - 1u;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    NsWriteSmem &S = *reinterpret_cast<NsWriteSmem *>(smem_raw);
    NsTiles &T = S.T;
    uint32_t(&wh)[kSortWarps][kRadix] = S.wh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = cdiv(n02, kSpTile);
    const uint64_t limit = wait_limit_ns();
    BulkPairLoader<int32_t, uint64_t, kSpTile> ld(T, SAR, Ax, n02);
    int64_t tile = blockIdx.x;
    if (tid == 0) ld.issue(tile, 0);
    for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const int64_t nxt = tile + gridDim.x;
        if (tid == 0 && nxt < ntiles) ld.issue(nxt, b ^ 1);
        for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&wh[0][0])[i] = 0;
        const bool whole = ld.whole(tile);
        const bool ok = ld.wait(tile, b, limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, 0, LOR_ERR_TIMEOUT);
                ld.drain(tile, b, nxt, limit);
            }
            __syncthreads();
            return;
        }
        const int wloc = warp * (kSpItems * 32) + lane;
        const int64_t wbase = tile * kSpTile + wloc;
        int32_t xs[kSpItems];
        uint64_t ws[kSpItems];
        uint32_t dig[kSpItems], r[kSpItems];
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) {
            const int64_t idx = wbase + i * 32;
            xs[i] = -1;
            ws[i] = 0;
            if (whole) {
                xs[i] = T.a[b][wloc + i * 32];
                ws[i] = T.b[b][wloc + i * 32];
            } else if (idx < n02) {
                xs[i] = SAR[idx];
                ws[i] = Ax[idx];
            }
            dig[i] = kNone;
            if (xs[i] >= 0 && xs[i] < n0) {
                dig[i] = uint32_t(ws[i] >> 40) & kMask;
            } else if (idx < n02 && (xs[i] < 0 || xs[i] >= n02)) {
                atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
            }
        }
        uint32_t *h = wh[warp];
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) r[i] = warp_peers_bits<kSymBits + 1>(dig[i]);
        const uint32_t lt_mask = lanemask_lt();
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) {
            const uint32_t d = dig[i];
            const uint32_t peers = r[i];
            const uint32_t lt = __popc(peers & lt_mask);
            const uint32_t c = d < kNone ? h[d] : 0u;
            r[i] = c + lt;
            __syncwarp();
            if (d < kNone && lt == 0) h[d] = c + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            // per digit: the counts of the warps before, plus the tile's start
            const int d = tid;
            uint32_t run = start[tile * kRadix + d];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = wh[w][d];
                wh[w][d] = run;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kSpItems; ++i) {
            if (dig[i] >= kNone) continue;
            const uint32_t o = wh[warp][dig[i]] + r[i];
            if (int64_t(o) >= n0) {  // counts that did not match SAR
                atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
                continue;
            }
            BRec16 v;
            v.t = xs[i];
            v.c01 = dig[i] | ((uint32_t(ws[i] >> 32) & 0xFFu) << 8);
            v.r1 = int32_t(wbase + i * 32 + 1);
            v.r2 = int32_t(uint32_t(ws[i]));
            out[o] = v;
        }
        __syncthreads();  // the warp counts and the buffer are reused by the next tile
    }
}

// ---- the level-0 merge on packed keys
//
// With both orders carried in sequence (Ax, Bx) the merge reads no records at
// random, and its cost is the in-tile merge-path search.  At level 0 every
// comparison key fits one 64-bit integer: a B1 sample p (and a nonsample, for
// that comparison) is (t_p << 32 | rank(S_p+1)), a B2 sample p (and a
// nonsample) is (t_p << 40 | t_p+1 << 32 | rank(S_p+2)); symbols are bytes and
// ranks fit 31 bits.  A sample's key carries its class in bit 63, a nonsample
// keeps both keys, and "sample before nonsample" is one integer comparison.
constexpr uint64_t kClass2 = uint64_t(1) << 63;

__device__ __forceinline__ bool ka_less(uint64_t ka, uint64_t kb1, uint64_t kb2) {
    return (ka & kClass2) ? (ka & ~kClass2) < kb2 : ka < kb1;
}

template <int kMergeItems>
__global__ void __launch_bounds__(kMergeTile / kMergeItems) k_merge_packed(MergeIn<uint8_t> a,
                                                                           const int64_t *__restrict__ split,
                                                                           int32_t *__restrict__ out, int *status) {
    constexpr int kMergeThreads = kMergeTile / kMergeItems;
    __shared__ uint64_t KA[kMergeTile];
    __shared__ ulonglong2 KB[kMergeTile];  // a nonsample's two keys, read together
    __shared__ int32_t PA[kMergeTile], PB[kMergeTile];
    const int64_t t = blockIdx.x;
    const int64_t tot = a.na + a.nb;
    const int64_t d0 = t * kMergeTile;
    const int64_t d1 = d0 + kMergeTile < tot ? d0 + kMergeTile : tot;
    int64_t a0 = split[t], a1 = split[t + 1];
    const int64_t a0c = min64(max64(a0, max64(0, d0 - a.nb)), min64(d0, a.na));
    int64_t a1c = min64(max64(a1, max64(0, d1 - a.nb)), min64(d1, a.na));
    a1c = min64(max64(a1c, a0c), a0c + (d1 - d0));
    if ((a0c != a0 || a1c != a1) && threadIdx.x == 0) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
    a0 = a0c;
    a1 = a1c;
    const int64_t b0 = d0 - a0, b1 = d1 - a1;
    const int na = int(a1 - a0), nb = int(b1 - b0), nt = int(d1 - d0);
    // Every slot's input is loaded before any is used, so that a thread keeps
    // all its loads in flight: a sample's index and key word, or a
    // nonsample's 16-byte record, in the same four registers.
    uint4 in[kMergeItems];
#pragma unroll
    for (int k = 0; k < kMergeItems; ++k) {
        const int sl = int(threadIdx.x) + k * kMergeThreads;
        in[k] = make_uint4(0u, 0u, 0u, 0u);
        if (sl < na) {
            const uint64_t w = a.Ax[a0 + sl];
            in[k] = make_uint4(uint32_t(a.A[a0 + sl]), uint32_t(w), uint32_t(w >> 32), 0u);
        } else if (sl < nt) {
            const BRec16 g = a.Bx[b0 + sl - na];
            in[k] = make_uint4(uint32_t(g.t), g.c01, uint32_t(g.r1), uint32_t(g.r2));
        }
    }
#pragma unroll
    for (int k = 0; k < kMergeItems; ++k) {
        const int sl = int(threadIdx.x) + k * kMergeThreads;
        if (sl < na) {
            const int32_t r = int32_t(in[k].x);
            const uint64_t rk = in[k].y, c0 = in[k].z & 0xFFu, c1 = (in[k].z >> 8) & 0xFFu;
            if (r < a.n0) {
                KA[sl] = (c0 << 32) | rk;
                PA[sl] = 3 * r + 1;
            } else {
                KA[sl] = kClass2 | (c0 << 40) | (c1 << 32) | rk;
                PA[sl] = 3 * (r - a.n0) + 2;
            }
        } else if (sl < nt) {
            const uint64_t c0 = in[k].y & 0xFFu, c1 = (in[k].y >> 8) & 0xFFu;
            KB[sl - na] = make_ulonglong2((c0 << 32) | uint64_t(in[k].z), (c0 << 40) | (c1 << 32) | uint64_t(in[k].w));
            PB[sl - na] = 3 * int32_t(in[k].x);
        }
    }
    __syncthreads();
    const int dl = min(int(threadIdx.x) * kMergeItems, nt);
    int lo = max(0, dl - nb), hi = min(dl, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int j = dl - 1 - mid;
        const ulonglong2 kb = KB[j];
        if (ka_less(KA[mid], kb.x, kb.y)) lo = mid + 1;
        else hi = mid;
    }
    int ia = lo, ib = dl - lo;
    int32_t o[kMergeItems];
#pragma unroll
    for (int k = 0; k < kMergeItems; ++k) {
        if (dl + k >= nt) break;
        bool take_a = ib >= nb;
        if (!take_a && ia < na) {
            const ulonglong2 kb = KB[ib];
            take_a = ka_less(KA[ia], kb.x, kb.y);
        }
        o[k] = take_a ? PA[ia++] : PB[ib++];
    }
    __syncthreads();  // the key arrays are dead: reuse PA as the output staging
#pragma unroll
    for (int k = 0; k < kMergeItems; ++k)
        if (dl + k < nt) PA[dl + k] = o[k];
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += kMergeThreads) out[d0 + i] = PA[i];
}

template <typename CharT>
__device__ __forceinline__ int64_t sym(const CharT *s, int64_t n, int64_t q) {
    return q < n ? int64_t(s[q]) : 0;
}

// ---- Step 1 by dense naming: when the key space is small the name of a key
// is 1 + the number of distinct keys below it, read from a table of present
// keys; no sort is needed unless the names come out unique.

// Small tables (level 0) are marked in shared memory first: thousands of
// blocks storing to the same few table lines would serialise in L2.
constexpr int kDenseLocal = 4096;

template <typename CharT, bool kValidate>
__global__ void __launch_bounds__(256) k_dense_mark(const CharT *__restrict__ s, int64_t n, int64_t n0,
                                                    int64_t n02, int kchars, uint32_t radix, int64_t maxc,
                                                    int64_t T, uint32_t *__restrict__ table, int *status) {
    __shared__ uint8_t seen[kDenseLocal];
    const bool local = T <= kDenseLocal;
    if (local)
        for (int i = threadIdx.x; i < T; i += blockDim.x) seen[i] = 0;
    __syncthreads();
    bool bad = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n02; j += stride) {
        const int64_t p = sample_pos(j, n0);
        uint32_t key = 0;
        for (int t = 0; t < kchars; ++t) {
            int64_t c = sym(s, n, p + t);
            if (p + t < n && (c < 1 || c > maxc)) {  // keeps the key inside the table
                bad = true;
                c = c < 1 ? 1 : maxc;
            }
            key = key * radix + uint32_t(c);
        }
        if (local) seen[key] = 1;
        else if (table[key] == 0u) table[key] = 1u;
    }
    if (kValidate && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t c = int64_t(s[0]);
        if (c < 1 || c > maxc) bad = true;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < T; i += blockDim.x)
            if (seen[i]) table[i] = 1u;
    }
}

// In place: table[k] = (present ? 1 + number of present keys below k : 0).
__global__ void __launch_bounds__(kScanThreads) k_dense_scan(uint32_t *__restrict__ table, int64_t m,
                                                             uint32_t *n_names, uint64_t *lb,
                                                             unsigned long long *ctr,
                                                             unsigned long long tile_base,
                                                             uint32_t epoch, int *status,
                                                             int64_t ntiles) {
    tile_compact(
        m, [&](int64_t k) { return table[k] != 0u; },
        [&](int64_t k, uint32_t o) { table[k] = o + 1; }, lb, ctr, tile_base, epoch, status, n_names,
        ntiles);
}

template <typename CharT>
__global__ void k_dense_write(const CharT *__restrict__ s, int64_t n, int64_t n0, int64_t n02, int kchars,
                              uint32_t radix, int64_t maxc, const uint32_t *__restrict__ table,
                              int32_t *__restrict__ R) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n02) return;
    const int64_t p = sample_pos(j, n0);
    uint32_t key = 0;
    for (int t = 0; t < kchars; ++t) {
        int64_t c = sym(s, n, p + t);
        if (p + t < n) c = c < 1 ? 1 : (c > maxc ? maxc : c);
        key = key * radix + uint32_t(c);
    }
    R[j] = int32_t(table[key]);
}

// Unique names are ranks: the sorted order is their inverse.
__global__ void k_dense_sorted(const int32_t *__restrict__ R, int64_t n02, int32_t *__restrict__ SAR,
                               int32_t *__restrict__ NS, int *status) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n02) return;
    const int32_t r = R[j];
    if (r < 1 || r > n02) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    SAR[r - 1] = int32_t(j);
    NS[r - 1] = r;
}

// ---- Step 1 from the parent's order: the parent level sorted every position
// of this level's string by its symbol (its name), so filtering that order to
// the sample positions sorts the samples by their first symbol; only runs of
// equal first symbols need their next two symbols.

__global__ void __launch_bounds__(kScanThreads) k_par_samples(
    const int32_t *__restrict__ PS, const int32_t *__restrict__ NS, int64_t n, int64_t n0, int dummy,
    uint32_t *__restrict__ SL, uint32_t *__restrict__ PRI, uint64_t *__restrict__ SEC, uint64_t *lb,
    unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch, int *status) {
    if (dummy && blockIdx.x == 0 && threadIdx.x == 0) {
        SL[0] = uint32_t(n0 - 1);  // the dummy position n, key (0,0,0): first
        PRI[0] = 0;
        SEC[0] = 0;
    }
    tile_compact(
        n, [&](int64_t j) { return PS[j] % 3 != 0; },
        [&](int64_t j, uint32_t o) {
            const int32_t x = PS[j];
            const int64_t slot = o + dummy;
            SL[slot] = x % 3 == 1 ? uint32_t((x - 1) / 3) : uint32_t(n0 + (x - 2) / 3);
            PRI[slot] = uint32_t(NS[j]);
            SEC[slot] = 0;
        },
        lb, ctr, tile_base, epoch, status, nullptr, 0);
}

__device__ __forceinline__ bool in_dup_run(const uint32_t *PRI, int64_t m, int64_t o) {
    const uint32_t v = PRI[o];
    return (o > 0 && PRI[o - 1] == v) || (o + 1 < m && PRI[o + 1] == v);
}

template <typename CharT>
__device__ __forceinline__ uint64_t second_third(const CharT *s, int64_t n, int64_t x, int bits) {
    return (uint64_t(sym(s, n, x + 1)) << bits) | uint64_t(sym(s, n, x + 2));
}

template <typename CharT>
__global__ void __launch_bounds__(kScanThreads) k_par_dups(
    const uint32_t *__restrict__ SL, const uint32_t *__restrict__ PRI, int64_t m, const CharT *__restrict__ s,
    int64_t n, int64_t n0, int bits, uint32_t *__restrict__ Dslot, uint32_t *__restrict__ Dsl,
    uint64_t *__restrict__ Dkey, uint32_t *count, uint64_t *lb, unsigned long long *ctr,
    unsigned long long tile_base, uint32_t epoch, int *status, int64_t ntiles) {
    tile_compact(
        m, [&](int64_t o) { return in_dup_run(PRI, m, o); },
        [&](int64_t o, uint32_t d) {
            const uint32_t j = SL[o];
            Dslot[d] = uint32_t(o);
            Dsl[d] = j;
            Dkey[d] = second_third(s, n, sample_pos(j, n0), bits);
        },
        lb, ctr, tile_base, epoch, status, count, ntiles);
}

// key32[i] = PRI[slot[v[i]]]: the first symbol of a duplicate, in the order
// of the previous (secondary) sort.
__global__ void k_gather_pri(const uint32_t *__restrict__ v, int64_t m, const uint32_t *__restrict__ slot,
                             const uint32_t *__restrict__ PRI, uint32_t *__restrict__ key32) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) key32[i] = PRI[slot[v[i]]];
}

// The sorted duplicates go back into the duplicate slots in slot order.
template <typename CharT>
__global__ void k_par_dup_writeback(const uint32_t *__restrict__ v, int64_t m,
                                    const uint32_t *__restrict__ Dslot, const uint32_t *__restrict__ Dsl,
                                    const CharT *__restrict__ s, int64_t n, int64_t n0, int bits,
                                    uint32_t *__restrict__ SL, uint64_t *__restrict__ SEC) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t d = v[i];
    const uint32_t o = Dslot[i];
    const uint32_t j = Dsl[d];
    SL[o] = j;
    SEC[o] = second_third(s, n, sample_pos(j, n0), bits);
}

__global__ void __launch_bounds__(kScanThreads) k_par_name(
    const uint32_t *__restrict__ SL, const uint32_t *__restrict__ PRI, const uint64_t *__restrict__ SEC,
    int64_t m, int32_t *__restrict__ R, int32_t *__restrict__ SAR, int32_t *__restrict__ NS,
    uint32_t *n_names, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base,
    uint32_t epoch, int *status) {
    tile_names(
        m, [&](int64_t o) { return o == 0 || PRI[o] != PRI[o - 1] || SEC[o] != SEC[o - 1]; },
        [&](int64_t o, uint32_t name) {
            const uint32_t j = SL[o];
            if (R) R[j] = int32_t(name);
            SAR[o] = int32_t(j);
            NS[o] = int32_t(name);
        },
        n_names, lb, ctr, tile_base, epoch, status);
}

// ---- Step 2 from the parent's order: nonsample positions 3t sorted by their
// symbol, then runs of equal symbols refined by rank(S_3t+1).

__global__ void __launch_bounds__(kScanThreads) k_par_nonsamples(
    const int32_t *__restrict__ PS, const int32_t *__restrict__ NS, int64_t n, uint32_t *__restrict__ T0,
    uint32_t *__restrict__ P0, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base,
    uint32_t epoch, int *status) {
    tile_compact(
        n, [&](int64_t j) { return PS[j] % 3 == 0; },
        [&](int64_t j, uint32_t o) {
            T0[o] = uint32_t(PS[j] / 3);
            P0[o] = uint32_t(NS[j]);
        },
        lb, ctr, tile_base, epoch, status, nullptr, 0);
}

__global__ void __launch_bounds__(kScanThreads) k_par_ns_dups(
    const uint32_t *__restrict__ T0, const uint32_t *__restrict__ P0, int64_t m,
    const int32_t *__restrict__ rankR, uint32_t *__restrict__ Dslot, uint32_t *__restrict__ Dt,
    uint32_t *__restrict__ Dkey, uint32_t *count, uint64_t *lb, unsigned long long *ctr,
    unsigned long long tile_base, uint32_t epoch, int *status, int64_t ntiles) {
    tile_compact(
        m, [&](int64_t o) { return in_dup_run(P0, m, o); },
        [&](int64_t o, uint32_t d) {
            const uint32_t t = T0[o];
            Dslot[d] = uint32_t(o);
            Dt[d] = t;
            Dkey[d] = uint32_t(rankR[t]);  // rank(S_3t+1)
        },
        lb, ctr, tile_base, epoch, status, count, ntiles);
}

__global__ void k_par_ns_writeback(const uint32_t *__restrict__ v, int64_t m, const uint32_t *__restrict__ Dslot,
                                   const uint32_t *__restrict__ Dt, uint32_t *__restrict__ T0) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) T0[Dslot[i]] = Dt[v[i]];
}

// ---------------------------------------------------------------- host driver

// ---- Prefix doubling on a reduced string whose names are almost unique
//
// When a level's names leave only a few samples sharing a name, the suffix
// array of its reduced string R follows from the name order by prefix
// doubling over the groups of equal names instead of one more DC3 level (the
// result is the same suffix array of R).  The rank of an R-suffix is one
// plus the index of the first element of its group in the current order.
// The pass with step h orders every unresolved group by (rank(j),
// rank(j + h)), rank 0 past the end of R, after which the order is by the
// first 2h symbols of R; a group of one is final.

// headof[v] = 1 + index of the first sample named v in name order.
__global__ void k_dbl_headof(const int32_t *__restrict__ NS, int64_t m, int32_t *__restrict__ headof) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < m && (k == 0 || NS[k] != NS[k - 1])) headof[NS[k]] = int32_t(k + 1);
}

// R[j] = rank of R-suffix j by its first symbol.
__global__ void k_dbl_init(int32_t *__restrict__ R, int64_t m, const int32_t *__restrict__ headof) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < m) R[j] = headof[R[j]];
}

// Positions (in name order) of samples that share their name.  Each thread
// loads its run of names with 16-byte loads, plus one name on either side.
// Persistent, like k_name.
__global__ void __launch_bounds__(kScanThreads) k_dbl_unresolved(
    const int32_t *__restrict__ NS, int64_t m, uint32_t *__restrict__ ul, uint32_t *count, uint64_t *lb,
    unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch, int *status, int64_t ntiles) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    const int64_t nt = ntiles > 0 ? ntiles : 1;  // an empty input still takes one (empty) tile
    for (;;) {
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= nt) break;  // uniform over the block
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    int32_t v[kScanItems];
    load_run<int32_t, kScanItems>(NS, base, m, -1, v);
    const int32_t before = base > 0 && base - 1 < m ? NS[base - 1] : -1;
    const int32_t after = base + kScanItems < m ? NS[base + kScanItems] : -2;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int32_t prev = i > 0 ? v[i - 1] : before;
        const int32_t next = i + 1 < kScanItems ? v[i + 1] : after;
        const bool in = base + i < m && (prev == v[i] || (base + i + 1 < m && next == v[i]));
        flags |= uint32_t(in) << i;
        cnt += in ? 1u : 0u;
    }
    uint32_t agg;
    const uint32_t excl = block_excl_scan<kScanThreads>(cnt, scratch, &agg);
    if (tid < 32) {
        const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
        if (tid == 0) {
            s_prefix = p;
            if (count && tile == ntiles - 1) *count = p + agg;
        }
    }
    __syncthreads();
    uint32_t o = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if ((flags >> i) & 1u) ul[o++] = uint32_t(base + i);
    __syncthreads();  // s_tile and s_prefix are reused by the next tile
    }
}

__global__ void k_dbl_keys(const uint32_t *__restrict__ ul, int64_t U, const int32_t *__restrict__ SAR,
                           const int32_t *__restrict__ R, int64_t m, int64_t h, int shift,
                           uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= U) return;
    const int32_t j = SAR[ul[i]];
    const uint32_t r2 = j + h < m ? uint32_t(R[j + h]) : 0u;
    key[i] = (uint64_t(uint32_t(R[j])) << shift) | r2;
    val[i] = uint32_t(j);
}

// Sorted unresolved samples go back to their slots; run ids and run starts
// of the refined groups.
__global__ void __launch_bounds__(kScanThreads) k_dbl_runs(
    const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, const uint32_t *__restrict__ ul,
    int64_t U, int32_t *__restrict__ SAR, uint32_t *__restrict__ runid, uint32_t *__restrict__ rstart,
    uint32_t *n_runs, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch,
    int *status) {
    tile_names(
        U, [&](int64_t i) { return i == 0 || key[i] != key[i - 1]; },
        [&](int64_t i, uint32_t r) {
            SAR[ul[i]] = int32_t(val[i]);
            runid[i] = r;
            if (i == 0 || key[i] != key[i - 1]) rstart[r - 1] = uint32_t(i);
        },
        n_runs, lb, ctr, tile_base, epoch, status);
}

__global__ void k_dbl_rank(const uint32_t *__restrict__ val, const uint32_t *__restrict__ runid,
                           const uint32_t *__restrict__ rstart, const uint32_t *__restrict__ ul, int64_t U,
                           int32_t *__restrict__ R) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < U) R[val[i]] = int32_t(ul[rstart[runid[i] - 1]] + 1);
}

// Samples whose refined group still holds more than one.
__global__ void __launch_bounds__(kScanThreads) k_dbl_next(
    const uint32_t *__restrict__ runid, const uint32_t *__restrict__ ul, int64_t U, uint32_t *__restrict__ ul2,
    uint32_t *count, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch,
    int *status, int64_t ntiles) {
    tile_compact(
        U,
        [&](int64_t i) {
            const uint32_t r = runid[i];
            return (i > 0 && runid[i - 1] == r) || (i + 1 < U && runid[i + 1] == r);
        },
        [&](int64_t i, uint32_t d) { ul2[d] = ul[i]; }, lb, ctr, tile_base, epoch, status, count, ntiles);
}

// The rest of the doubling in one block once few samples are unresolved:
// every pass of the loop above (keys, sort, run ranks, next unresolved set)
// on a shared-memory copy of the unresolved list, sorted by a block bitonic
// sort, until no group holds more than one sample.  Keys of a pass are all
// read before any rank of that pass is written, as in the multi-kernel loop.
constexpr int kDblSmall = 4096;
constexpr int kDblSmallThreads = 1024;
constexpr int kDblSmallRounds = 40;

struct DblSmallSmem {
    uint64_t key[kDblSmall];
    uint32_t val[kDblSmall];
    uint32_t ul[kDblSmall];
    uint32_t run[kDblSmall];    // run id (1-based) of each sorted element
    uint32_t rstart[kDblSmall];  // first element of each run
    uint32_t scratch[kDblSmallThreads / 32 + 1];
    uint32_t count;
};

// When skip_big is set an unresolved set larger than kDblSmall is left for
// the multi-kernel rounds (no error); a finished set zeroes *U_in.
__global__ void __launch_bounds__(kDblSmallThreads) k_dbl_small(const uint32_t *__restrict__ ul_in,
                                                                uint32_t *U_in, int64_t m, int64_t h0,
                                                                int shift, int32_t *__restrict__ SAR,
                                                                int32_t *__restrict__ R, int *status,
                                                                int skip_big) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DblSmallSmem &S = *reinterpret_cast<DblSmallSmem *>(smem_raw);
    const int tid = threadIdx.x;
    constexpr int kPer = kDblSmall / kDblSmallThreads;
    int U = int(*U_in);
    if (U > kDblSmall) {
        if (tid == 0 && !skip_big) atomicCAS(status, 0, LOR_ERR_INVALID_ARG);
        return;
    }
    if (U == 0) return;
    for (int i = tid; i < U; i += kDblSmallThreads) S.ul[i] = ul_in[i];
    __syncthreads();
    int64_t h = h0;
    for (int round = 0; U > 0; ++round, h *= 2) {
        if (h >= m || round >= kDblSmallRounds) {  // cannot happen for a valid R
            if (tid == 0) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
            return;
        }
        int P = 1;
        while (P < U) P <<= 1;
        for (int i = tid; i < P; i += kDblSmallThreads) {
            if (i < U) {
                const int32_t j = SAR[S.ul[i]];
                const uint32_t r2 = j + h < m ? uint32_t(R[j + h]) : 0u;
                S.key[i] = (uint64_t(uint32_t(R[j])) << shift) | r2;
                S.val[i] = uint32_t(j);
            } else {
                S.key[i] = ~uint64_t(0);
                S.val[i] = 0;
            }
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = tid; i < P; i += kDblSmallThreads) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const uint64_t a = S.key[i], b = S.key[l];
                        if ((a > b) == up) {
                            S.key[i] = b;
                            S.key[l] = a;
                            const uint32_t t = S.val[i];
                            S.val[i] = S.val[l];
                            S.val[l] = t;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // Run ids: blocked kPer items per thread, block scan of the run starts.
        uint32_t cnt = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int i = tid * kPer + q;
            if (i < U && (i == 0 || S.key[i] != S.key[i - 1])) cnt++;
        }
        uint32_t total;
        uint32_t r = block_excl_scan<kDblSmallThreads>(cnt, S.scratch, &total);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int i = tid * kPer + q;
            if (i < U) {
                if (i == 0 || S.key[i] != S.key[i - 1]) {
                    ++r;
                    S.rstart[r - 1] = uint32_t(i);
                }
                S.run[i] = r;
            }
        }
        __syncthreads();
        for (int i = tid; i < U; i += kDblSmallThreads) {
            SAR[S.ul[i]] = int32_t(S.val[i]);
            R[S.val[i]] = int32_t(S.ul[S.rstart[S.run[i] - 1]] + 1);
        }
        // Next unresolved set: members of runs with more than one element.
        cnt = 0;
        bool keep[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int i = tid * kPer + q;
            keep[q] = i < U && ((i > 0 && S.run[i - 1] == S.run[i]) || (i + 1 < U && S.run[i + 1] == S.run[i]));
            cnt += keep[q] ? 1u : 0u;
        }
        uint32_t o = block_excl_scan<kDblSmallThreads>(cnt, S.scratch, &total);
        uint32_t nxt[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) nxt[q] = keep[q] ? S.ul[tid * kPer + q] : 0u;
        __syncthreads();  // every old list entry is read before the list is rewritten
#pragma unroll
        for (int q = 0; q < kPer; ++q)
            if (keep[q]) S.ul[o++] = nxt[q];
        U = int(total);
        __syncthreads();
    }
    if (tid == 0) *U_in = 0;
}

// The doubling round kernels over a device-held unresolved count (graph
// mode): grid-stride or resident-block forms of the kernels above.
__global__ void k_dbl_keys_dev(const uint32_t *__restrict__ ul, const uint32_t *U_dev,
                               const int32_t *__restrict__ SAR, const int32_t *__restrict__ R, int64_t m,
                               int64_t h, int shift, uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t j = SAR[ul[i]];
        const uint32_t r2 = j + h < m ? uint32_t(R[j + h]) : 0u;
        key[i] = (uint64_t(uint32_t(R[j])) << shift) | r2;
        val[i] = uint32_t(j);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_dbl_runs_dev(
    const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, const uint32_t *__restrict__ ul,
    const uint32_t *U_dev, int32_t *__restrict__ SAR, uint32_t *__restrict__ runid,
    uint32_t *__restrict__ rstart, uint64_t *lb, unsigned long long *ctr, uint32_t epoch, int *status) {
    tile_names_dyn(
        U_dev, [&](int64_t i) { return i == 0 || key[i] != key[i - 1]; },
        [&](int64_t i, uint32_t r) {
            SAR[ul[i]] = int32_t(val[i]);
            runid[i] = r;
            if (i == 0 || key[i] != key[i - 1]) rstart[r - 1] = uint32_t(i);
        },
        lb, ctr, epoch, status);
}

__global__ void k_dbl_rank_dev(const uint32_t *__restrict__ val, const uint32_t *__restrict__ runid,
                               const uint32_t *__restrict__ rstart, const uint32_t *__restrict__ ul,
                               const uint32_t *U_dev, int32_t *__restrict__ R) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x)
        R[val[i]] = int32_t(ul[rstart[runid[i] - 1]] + 1);
}

__global__ void __launch_bounds__(kScanThreads) k_dbl_next_dev(
    const uint32_t *__restrict__ runid, const uint32_t *__restrict__ ul, const uint32_t *U_dev,
    uint32_t *__restrict__ ul2, uint32_t *count, uint64_t *lb, unsigned long long *ctr, uint32_t epoch,
    int *status) {
    const int64_t U = int64_t(*U_dev);
    tile_compact_dyn(
        U_dev,
        [&](int64_t i) {
            const uint32_t r = runid[i];
            return (i > 0 && runid[i - 1] == r) || (i + 1 < U && runid[i + 1] == r);
        },
        [&](int64_t i, uint32_t d) { ul2[d] = ul[i]; }, lb, ctr, epoch, status, count);
}

// Ranks of the samples that share their name, once every sample holds
// 1 + its position in name order (exact for the samples whose name is
// unique): in the unresolved list (name order, the members of every group of
// two or more) the first of each run of equal names is its group's head, and
// every member takes the head's rank.
__global__ void k_dbl_group_heads(const uint32_t *__restrict__ ul, const uint32_t *U_dev,
                                  const int32_t *__restrict__ NS, int32_t *__restrict__ headof) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t k = ul[i];
        const int32_t v = NS[k];
        if (i == 0 || NS[ul[i - 1]] != v) headof[v] = int32_t(k + 1);
    }
}
// The same from the names listed beside the unresolved positions.
__global__ void k_dbl_group_heads_named(const uint32_t *__restrict__ ul, const int32_t *__restrict__ names,
                                        const uint32_t *U_dev, int32_t *__restrict__ headof) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = names[i];
        if (i == 0 || names[i - 1] != v) headof[v] = int32_t(ul[i] + 1);
    }
}
// names[i] = NS[ul[i]] (the names beside the list, for the text round).
__global__ void k_dbl_list_names(const uint32_t *__restrict__ ul, const uint32_t *U_dev, const int32_t *__restrict__ NS,
                                 int32_t *__restrict__ names) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x)
        names[i] = NS[ul[i]];
}
__global__ void k_dbl_group_ranks(const uint32_t *__restrict__ ul, const uint32_t *U_dev,
                                  const int32_t *__restrict__ NS, const int32_t *__restrict__ SAR,
                                  const int32_t *__restrict__ headof, int32_t *__restrict__ R) {
    const int64_t U = int64_t(*U_dev);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t k = ul[i];
        R[SAR[k]] = headof[NS[k]];
    }
}

// After the last enqueued round nothing may be left unresolved.
__global__ void k_dbl_check_done(const uint32_t *U_dev, int *status) {
    if (threadIdx.x == 0 && *U_dev != 0) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
}

struct TraceRow {
    int64_t n, names;
    int32_t key_bits;
};
thread_local std::vector<TraceRow> g_trace;

// Route controls (lor_dc3_route_set): they pick how the sample is ordered,
// never what the suffix array is.
std::atomic<int> g_route_k0{0};        // symbols named at level 0 (0: 2-bit keys when the text allows, 1: from the key width)
std::atomic<int> g_route_strategy{0};  // 1: radix sort at every level
std::atomic<int> g_route_doubling{1};  // 0 never, 1 when names are almost unique, 2 whenever names repeat

// Symbols named at level 0: the longest prefix whose key, in base maxc + 1,
// fits the configured key width (48 bits by default: six 8-bit radix passes,
// 17 symbols for a DNA pair),
// so that on text without long repeats the names come out almost unique and
// the reduced string is finished by prefix doubling.  Naming by any prefix of
// at least 3 symbols keeps the order of the reduced string's suffixes equal
// to the order of the sample suffixes.  lor_dc3_route_set can force it.
int level0_kchars(int bits, int64_t maxc) {
    const int budget = tune_config().level0_key_bits;
    int k = 0;
    for (unsigned __int128 T = 1; k < kKeyMaxChars; ++k) {
        T *= uint64_t(maxc) + 1;
        if (T > (unsigned __int128)1 << budget) break;
    }
    if (k < 3) k = 3;
    const int forced = g_route_k0.load(std::memory_order_relaxed);
    if (forced >= 3) k = forced;
    const int kmax = 64 / (bits > 0 ? bits : 1);
    return k > kmax ? kmax : k;
}

struct Dc3Run {
    cudaStream_t s;
    int *status;
    char *ws;
    Dc3Layout L;
    RadixScratch rs;
    int doubling;       // 0 never, 1 when names are almost unique, 2 whenever names repeat
    uint32_t *d_names;  // count read back after naming
    uint32_t *d_count;  // count read back after a compaction
    uint64_t *t64[3];
    uint32_t *t32[6];
    uint32_t *tbl;
    bool force_lsd;
};

inline unsigned grid_for(int64_t m, int nt) { return unsigned(cdiv(m > 0 ? m : 1, nt)); }

int read_u32(Dc3Run &D, const uint32_t *d, uint32_t *h) {
    LOR_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, D.s));
    LOR_CUDA_TRY(cudaStreamSynchronize(D.s));
    return LOR_OK;
}

// Launch a tile_compact/tile_names kernel: claims its tiles from the running
// counter under a fresh look-back epoch.
#define LOR_TILE_LAUNCH(D, m, kernel, ...)                                                 \
    do {                                                                                  \
        const int64_t _nt = cdiv((m) > 0 ? (m) : 1, kScanTile);                           \
        (D).rs.epoch++;                                                                   \
        kernel<<<unsigned(_nt), kScanThreads, 0, (D).s>>>(__VA_ARGS__);                   \
        LOR_LAUNCH_CHECK();                                                               \
        (D).rs.tile_base += (unsigned long long)_nt;                                      \
    } while (0)

// The same for a persistent tile kernel: a resident grid claims tiles until
// each block draws one past the end, so the launch makes ntiles + grid claims.
#define LOR_PTILE_LAUNCH(D, m, kernel, ...)                                                \
    do {                                                                                  \
        const int64_t _nt = cdiv((m) > 0 ? (m) : 1, kScanTile);                           \
        const unsigned _g = unsigned(min64(_nt, int64_t(scan_grid_cap())));               \
        (D).rs.epoch++;                                                                   \
        kernel<<<_g, kScanThreads, 0, (D).s>>>(__VA_ARGS__);                              \
        LOR_LAUNCH_CHECK();                                                               \
        (D).rs.tile_base += (unsigned long long)_nt + _g;                                 \
    } while (0)

#define LB_ARGS(D) (D).rs.lookback, (D).rs.tile_ctr, (D).rs.tile_base, (D).rs.epoch, (D).status

// Inputs of at least this many entries scatter through bucketing.
constexpr int64_t kBucketMin = int64_t(1) << 22;

// rankR[SAR[j]] = j + 1 (the inverse of the level below's suffix array).
int rank_scatter(Dc3Run &D, const int32_t *SAR, int64_t m, int32_t *Rl) {
    if (m < kBucketMin || D.force_lsd) {
        ProfScope ps(PK_RANK_SCATTER, double(m) * 8, D.s);
        k_rank_scatter<<<grid_for(m, 256), 256, 0, D.s>>>(SAR, m, Rl, D.status);
        LOR_LAUNCH_CHECK();
        return LOR_OK;
    }
    return bucketed_scatter(D.rs, (const uint32_t *)SAR, nullptr, m, m, (uint32_t *)D.t64[0], D.t32[0],
                            D.t32[1], Rl, 1);
}

inline bool bucket_names(const Dc3Run &D, const LevelSizes &z) { return z.n02 >= kBucketMin && !D.force_lsd; }

// R[SAR[j]] = NS[j]: the names in reduced-string order, for naming kernels
// that left R unwritten (large levels).
int names_scatter(Dc3Run &D, const int32_t *SAR, const int32_t *NSl, int64_t m, int32_t *Rl) {
    return bucketed_scatter(D.rs, (const uint32_t *)SAR, (const uint32_t *)NSl, m, m, D.t32[2], D.t32[3],
                            D.t32[4], Rl, 0);
}

// ---- Step 1, strategy "sort": LSD radix sort of the keys, then naming.
template <typename CharT, typename KeyT>
int sample_sort_and_name(Dc3Run &D, int lvl, const CharT *s, const LevelSizes &z, int kchars,
                         int key_bits, int64_t maxc, int32_t *Rl, int32_t *SAR, int32_t *NSl) {
    const uint64_t radix = uint64_t(maxc) + 1;
    cudaStream_t st = D.s;
    KeyT *k0 = (KeyT *)D.t64[0], *k1 = (KeyT *)D.t64[1];
    bool hist_ready = false;
    if constexpr (sizeof(CharT) == 1) {
        // Level 0: staged keys with the digit histograms counted on the way.
        const int dbits = tune_config().digit_bits;
        const int npasses = int(cdiv(key_bits, dbits));
        if (kchars > kKeyMaxChars || npasses > kMaxPasses) return LOR_ERR_INVALID_ARG;
        LOR_CUDA_TRY(cudaMemsetAsync(D.rs.hist, 0, sizeof(uint32_t) * kMaxPasses * kRadix, st));
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * sizeof(KeyT) + double(z.n), st);
        const dim3 grid(unsigned(cdiv(max64(z.n0, z.n2), kKeyTile)), 2);
        int chunk = 1;
        for (uint64_t T = radix; T * radix <= (uint64_t(1) << 32); T *= radix) ++chunk;
        k_sample_keys0<KeyT><<<grid, 256, 0, st>>>(s, z.n, z.n0, z.n2, kchars, chunk, uint32_t(radix), maxc, k0,
                                                   npasses, key_bits, dbits, D.rs.hist, D.status);
        hist_ready = true;
    } else {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * (sizeof(KeyT) + 4.0 * kchars / 3.0), st);
        k_sample_keys<CharT, KeyT, false><<<grid_for(z.n02, 256), 256, 0, st>>>(
            s, z.n, z.n0, z.n02, 0, kchars, radix, maxc, k0, D.status);
    }
    LOR_LAUNCH_CHECK();
    KeyT *kr;
    uint32_t *vr;
    // Level 0: samples with equal keys get one name, and neither the doubling
    // that resolves them nor the recursion reads their order, so the first
    // pass need not be stable.
    int rc = radix_sort_pairs<KeyT>(D.rs, k0, D.t32[0], k1, D.t32[1], z.n02, 0, key_bits, true, &kr, &vr,
                                    hist_ready, nullptr, sizeof(CharT) == 1);
    if (rc) return rc;
    {
        ProfScope ps(PK_NAMING, double(z.n02) * (sizeof(KeyT) + 16), st);
        LOR_PTILE_LAUNCH(D, z.n02, k_name<KeyT>, kr, vr, z.n02, bucket_names(D, z) ? nullptr : Rl, SAR, NSl,
                        D.d_names, LB_ARGS(D));
    }
    return LOR_OK;  // large levels: R is written by dc3_level once it knows how to continue
}

// Triples too wide for 64 bits: stable sort by (t_i+1, t_i+2), then by t_i.
template <typename CharT>
int sample_sort_and_name_wide(Dc3Run &D, const CharT *s, const LevelSizes &z, int bits, int64_t maxc,
                              int32_t *Rl, int32_t *SAR, int32_t *NSl) {
    cudaStream_t st = D.s;
    uint64_t *k0 = D.t64[0], *k1 = D.t64[1];
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * (8 + 8), st);
        k_sample_keys<CharT, uint64_t, false><<<grid_for(z.n02, 256), 256, 0, st>>>(
            s, z.n, z.n0, z.n02, 1, 3, uint64_t(maxc) + 1, maxc, k0, D.status);
    }
    LOR_LAUNCH_CHECK();
    uint64_t *kr;
    uint32_t *vr;
    const int pair_bits = bit_width_u64((uint64_t(maxc) + 1) * (uint64_t(maxc) + 1) - 1);
    int rc = radix_sort_pairs<uint64_t>(D.rs, k0, D.t32[0], k1, D.t32[1], z.n02, 0, pair_bits, true, &kr, &vr);
    if (rc) return rc;
    uint32_t *kx = (uint32_t *)(kr == k0 ? k1 : k0);  // free key buffer
    uint32_t *ky = (uint32_t *)kr;
    uint32_t *vx = vr, *vy = (vr == D.t32[0] ? D.t32[1] : D.t32[0]);
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * (4 + 4 + 4), st);
        k_first_char<CharT><<<grid_for(z.n02, 256), 256, 0, st>>>(vx, z.n02, s, z.n, z.n0, kx);
    }
    LOR_LAUNCH_CHECK();
    uint32_t *kr2, *vr2;
    rc = radix_sort_pairs<uint32_t>(D.rs, kx, vx, ky, vy, z.n02, 0, bits, false, &kr2, &vr2);
    if (rc) return rc;
    {
        ProfScope ps(PK_NAMING, double(z.n02) * (4 + 12 + 12 * 2), st);
        LOR_TILE_LAUNCH(D, z.n02, k_name_gather<CharT>, vr2, z.n02, s, z.n, z.n0,
                        bucket_names(D, z) ? nullptr : Rl, SAR, NSl, D.d_names, LB_ARGS(D));
    }
    return LOR_OK;  // large levels: R is written by dc3_level once it knows how to continue
}

// ---- Step 1 at level 0 for DNA texts: 16-symbol keys at 2 bits a symbol
// (dc3_packed.cuh): a counting pre-pass over the text, one partition pass
// that makes the keys as it goes, three stable passes on (u32, u32) pairs,
// the exception windows put in order, naming.  When the text has more
// exception windows than the fix-up can order, *used stays false and nothing
// a later route reads has been changed.
int sample_packed_sort_and_name(Dc3Run &D, const uint8_t *s, const LevelSizes &z, int64_t maxc, int32_t *Rl,
                                int32_t *SAR, int32_t *NSl, bool *used) {
    cudaStream_t st = D.s;
    *used = false;
    const int64_t m = z.n02;
    const uint32_t mc = uint32_t(maxc), lo = maxc > 4 ? uint32_t(maxc - 3) : 1u;
    uint32_t *exc_list = D.t32[4];  // at most m entries are written
    LOR_CUDA_TRY(cudaMemsetAsync(D.rs.hist, 0, sizeof(uint32_t) * kPkHistWords, st));
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n), st);
        const dim3 grid(unsigned(cdiv(max64(z.n0, z.n2), kPkTile)), 2);
        k_pk_count<<<grid, kPkThreads, 0, st>>>(s, z.n, z.n0, z.n2, mc, lo, D.rs.hist, exc_list, D.status);
    }
    LOR_LAUNCH_CHECK();
    k_pk_offsets<<<1, kRadix, 0, st>>>(D.rs.hist, D.rs.offsets);
    LOR_LAUNCH_CHECK();
    uint32_t hh[kPkHistWords];
    LOR_CUDA_TRY(cudaMemcpyAsync(hh, D.rs.hist, sizeof(hh), cudaMemcpyDeviceToHost, st));
    LOR_CUDA_TRY(cudaStreamSynchronize(st));
    const uint32_t nexc = hh[kPkExcCount];
    if (nexc > uint32_t(kPkExcMax)) return LOR_OK;
    *used = true;
    uint32_t *k0 = D.t32[0], *v0 = D.t32[1], *k1 = D.t32[2], *v1 = D.t32[3];
    {
        ProfScope ps(PK_RADIX_PASS, double(z.n) + double(m) * 8, st);
        const size_t smem = sizeof(PkPartSmem);
        LOR_CUDA_TRY(cudaFuncSetAttribute(k_pk_partition, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        const int64_t ntiles = cdiv(z.n0, kPkTile) + cdiv(z.n2, kPkTile);
        const unsigned grid = unsigned(min64(ntiles, sort_grid_cap()));
        k_pk_partition<<<grid, kPkThreads, smem, st>>>(s, z.n, z.n0, z.n2, mc, lo, k0, v0, D.rs.offsets + kPkHist0,
                                                      D.status);
    }
    LOR_LAUNCH_CHECK();
    uint32_t *kr, *vr;
    int rc = tune_config().sort_items_32 == 12
                 ? radix_passes<uint32_t, 12>(D.rs, k0, v0, k1, v1, m, 8, 32, 8, 3, hh, true, nullptr, &kr, &vr, false)
                 : radix_passes<uint32_t, 16>(D.rs, k0, v0, k1, v1, m, 8, 32, 8, 3, hh, true, nullptr, &kr, &vr, false);
    if (rc) return rc;
    if (nexc > 0) {
        ProfScope ps(PK_NAMING, double(nexc) * 48, st);
        const size_t smem = sizeof(PkFixSmem);
        LOR_CUDA_TRY(cudaFuncSetAttribute(k_pk_fixup, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_pk_fixup<<<1, 1024, smem, st>>>(s, z.n, z.n0, mc, lo, D.rs.hist, exc_list, kr, vr, m, D.status);
        LOR_LAUNCH_CHECK();
    }
    {
        ProfScope ps(PK_NAMING, double(m) * 16, st);
        // the unresolved list goes to t32[5] and its names to t64[2], which the
        // rank scatter leaves alone
        LOR_PTILE_LAUNCH(D, m, k_pk_name, kr, vr, m, s, z.n, z.n0, mc, bucket_names(D, z) ? nullptr : Rl, SAR, NSl,
                         D.d_names, D.t32[5], (int32_t *)D.t64[2], D.d_count, D.rs.lookback,
                         D.rs.lookback + cdiv(m, kScanTile), D.rs.tile_ctr, D.rs.tile_base, D.rs.epoch, D.status);
    }
    return LOR_OK;  // large levels: R is written by dc3_level once it knows how to continue
}

// ---- Step 1, strategy "dense": names from a table of present keys.
template <typename CharT>
int sample_dense_names(Dc3Run &D, int lvl, const CharT *s, const LevelSizes &z, int kchars, int64_t T,
                       int64_t maxc, int32_t *Rl, int32_t *SAR, int32_t *NSl, uint32_t *names) {
    cudaStream_t st = D.s;
    const uint32_t radix = uint32_t(maxc + 1);
    LOR_CUDA_TRY(cudaMemsetAsync(D.tbl, 0, sizeof(uint32_t) * size_t(T), st));
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * (kchars * sizeof(CharT) / 3.0 + 4), st);
        const unsigned grid = unsigned(min64(cdiv(z.n02, 256), 152 * 8));
        if (lvl == 0)
            k_dense_mark<CharT, true><<<grid, 256, 0, st>>>(s, z.n, z.n0, z.n02, kchars, radix, maxc, T,
                                                             D.tbl, D.status);
        else
            k_dense_mark<CharT, false><<<grid, 256, 0, st>>>(s, z.n, z.n0, z.n02, kchars, radix, maxc, T,
                                                              D.tbl, D.status);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_NAMING, double(T) * 8, st);
        const int64_t ntiles = cdiv(T, kScanTile);
        LOR_TILE_LAUNCH(D, T, k_dense_scan, D.tbl, T, D.d_names, LB_ARGS(D), ntiles);
    }
    {
        ProfScope ps(PK_NAMING, double(z.n02) * (kchars * sizeof(CharT) / 3.0 + 8), st);
        k_dense_write<CharT><<<grid_for(z.n02, 256), 256, 0, st>>>(s, z.n, z.n0, z.n02, kchars, radix, maxc,
                                                                   D.tbl, Rl);
    }
    LOR_LAUNCH_CHECK();
    int rc = read_u32(D, D.d_names, names);
    if (rc) return rc;
    if (int64_t(*names) == z.n02) {
        ProfScope ps(PK_RANK_SCATTER, double(z.n02) * 12, st);
        k_dense_sorted<<<grid_for(z.n02, 256), 256, 0, st>>>(Rl, z.n02, SAR, NSl, D.status);
        LOR_LAUNCH_CHECK();
    }
    return LOR_OK;
}

// Sort (key, value) pairs of a duplicate subset: by key (key_bits), then
// stably by the first symbol PRI[slot[v]] (pri_bits).  Returns the value
// order in *vout.
template <typename KeyT>
int sort_dups_then_by_first(Dc3Run &D, KeyT *keys, int64_t nd, int key_bits, const uint32_t *slot,
                            const uint32_t *PRI, int pri_bits, uint32_t **vout) {
    cudaStream_t st = D.s;
    KeyT *kalt = (KeyT *)D.t64[2];
    KeyT *kr;
    uint32_t *vr;
    int rc = radix_sort_pairs<KeyT>(D.rs, keys, D.t32[4], kalt, D.t32[5], nd, 0, key_bits, true, &kr, &vr);
    if (rc) return rc;
    uint32_t *kx = (uint32_t *)(kr == keys ? (void *)kalt : (void *)keys);
    uint32_t *ky = (uint32_t *)kr;
    uint32_t *vy = vr == D.t32[4] ? D.t32[5] : D.t32[4];
    k_gather_pri<<<grid_for(nd, 256), 256, 0, st>>>(vr, nd, slot, PRI, kx);
    LOR_LAUNCH_CHECK();
    uint32_t *kr2;
    rc = radix_sort_pairs<uint32_t>(D.rs, kx, vr, ky, vy, nd, 0, pri_bits, false, &kr2, vout);
    return rc;
}

// ---- Step 1, strategy "parent order".
template <typename CharT>
int sample_from_parent(Dc3Run &D, const CharT *s, const LevelSizes &z, int bits, const int32_t *PS,
                       const int32_t *PNS, int32_t *Rl, int32_t *SAR, int32_t *NSl, int64_t *dups) {
    cudaStream_t st = D.s;
    const int dummy = (z.n0 > z.n1) ? 1 : 0;
    uint32_t *SL = D.t32[0], *PRI = D.t32[1], *Dslot = D.t32[2], *Dsl = D.t32[3];
    uint64_t *SEC = D.t64[0], *Dkey = D.t64[1];
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n) * 8 + double(z.n02) * 16, st);
        LOR_TILE_LAUNCH(D, z.n, k_par_samples, PS, PNS, z.n, z.n0, dummy, SL, PRI, SEC, LB_ARGS(D));
    }
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(z.n02) * 8, st);
        const int64_t ntiles = cdiv(z.n02, kScanTile);
        LOR_TILE_LAUNCH(D, z.n02, k_par_dups<CharT>, SL, PRI, z.n02, s, z.n, z.n0, bits, Dslot, Dsl, Dkey,
                        D.d_count, LB_ARGS(D), ntiles);
    }
    uint32_t nd = 0;
    int rc = read_u32(D, D.d_count, &nd);
    if (rc) return rc;
    *dups = nd;
    if (nd > 0) {
        uint32_t *vord;
        rc = sort_dups_then_by_first<uint64_t>(D, Dkey, nd, 2 * bits, Dslot, PRI, bits, &vord);
        if (rc) return rc;
        k_par_dup_writeback<CharT><<<grid_for(nd, 256), 256, 0, st>>>(vord, nd, Dslot, Dsl, s, z.n, z.n0,
                                                                      bits, SL, SEC);
        LOR_LAUNCH_CHECK();
    }
    {
        ProfScope ps(PK_NAMING, double(z.n02) * (4 + 4 + 8 + 4 + 4 + 4), st);
        LOR_TILE_LAUNCH(D, z.n02, k_par_name, SL, PRI, SEC, z.n02, bucket_names(D, z) ? nullptr : Rl, SAR,
                        NSl, D.d_names, LB_ARGS(D));
    }
    return LOR_OK;  // large levels: R is written by dc3_level once it knows how to continue
}

struct TraceExtra {
    int strategy;  // 0 sort, 1 dense, 2 parent order, 3 prefix doubling
    int64_t dups;
};
thread_local std::vector<TraceExtra> g_trace_extra;

// Suffix array of the reduced string R (length m, names in R order in Rl,
// samples in name order in SAR with their names in NSl) by prefix doubling;
// leaves SA_R in SAR and rank(R-suffix) in Rl, like a returned recursion
// followed by the rank scatter.  *U0 receives the initial unresolved count.
// When ul_ready is set (D.t32[5]) the naming kernel has already listed the
// unresolved positions there, with their names in D.t64[2] and their count
// in D.d_count.  Level 0 passes
// its text (T0 != nullptr; names are the first kchars symbols of each
// sample): the groups of two are then settled on the text first.
struct Level0Text {
    const uint8_t *s = nullptr;
    int64_t n = 0, n0 = 0;
    uint32_t maxc = 0;
    int kchars = 0;
};

// Entries of the unresolved list whose group still holds more than one.
__global__ void __launch_bounds__(kScanThreads) k_dbl_keep(
    const uint32_t *__restrict__ keep, const uint32_t *__restrict__ ul, int64_t U, uint32_t *__restrict__ ul2,
    uint32_t *count, uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch,
    int *status, int64_t ntiles) {
    tile_compact(
        U, [&](int64_t i) { return keep[i] != 0; }, [&](int64_t i, uint32_t d) { ul2[d] = ul[i]; }, lb, ctr,
        tile_base, epoch, status, count, ntiles);
}

int sa_by_doubling(Dc3Run &D, int32_t *Rl, int64_t m, int32_t *SAR, const int32_t *NSl, bool r_unwritten,
                   int64_t *U0, bool ul_ready = false, const Level0Text *T0 = nullptr) {
    cudaStream_t st = D.s;
    int32_t *headof = (int32_t *)D.t32[0];
    uint32_t *ul = D.t32[1], *ul2 = D.t32[2], *runid = D.t32[3], *val = D.t32[4], *rstart = D.t32[5];
    if (ul_ready) {
        ul = D.t32[5];
        rstart = D.t32[1];
    }
    int32_t *ul_names = (int32_t *)D.t64[2];  // names beside the list (level 0's text round)
    uint32_t *valt = D.t32[0];  // headof is dead once the ranks are initialised
    uint64_t *k0 = D.t64[0], *k1 = D.t64[1];
    if (r_unwritten) {
        // Large levels left R unwritten: every sample first takes 1 + its
        // position in name order (an inverse-permutation scatter with the
        // values generated), then the members of the groups of equal names take
        // their group head's rank.
        int rc = bucketed_scatter(D.rs, (const uint32_t *)SAR, nullptr, m, m, D.t32[2], D.t32[3], D.t32[4], Rl, 1);
        if (rc) return rc;
    } else {
        {
            ProfScope ps(PK_NAMING, double(m) * 8, st);
            k_dbl_headof<<<grid_for(m, 256), 256, 0, st>>>(NSl, m, headof);
            LOR_LAUNCH_CHECK();
        }
        ProfScope ps(PK_NAMING, double(m) * 12, st);
        k_dbl_init<<<grid_for(m, 256), 256, 0, st>>>(Rl, m, headof);
        LOR_LAUNCH_CHECK();
    }
    if (!ul_ready) {
        ProfScope ps(PK_NAMING, double(m) * 8, st);
        const int64_t ntiles = cdiv(m, kScanTile);
        LOR_PTILE_LAUNCH(D, m, k_dbl_unresolved, NSl, m, ul, D.d_count, LB_ARGS(D), ntiles);
    }
    uint32_t hU = 0;
    int rc = read_u32(D, D.d_count, &hU);
    if (rc) return rc;
    *U0 = hU;
    if (T0 && hU > 0) {
        // groups of two settled on the text; larger groups take their head's
        // rank (large levels) and stay
        const unsigned g = unsigned(min64(cdiv(hU, 256), 152 * 8));
        if (r_unwritten) {
            ProfScope ps(PK_NAMING, double(hU) * 12, st);
            if (ul_ready) k_dbl_group_heads_named<<<g, 256, 0, st>>>(ul, ul_names, D.d_count, headof);
            else k_dbl_group_heads<<<g, 256, 0, st>>>(ul, D.d_count, NSl, headof);
            LOR_LAUNCH_CHECK();
        }
        if (!ul_ready) {
            // the names beside the list, for the text round
            ProfScope ps(PK_NAMING, double(hU) * 8, st);
            k_dbl_list_names<<<g, 256, 0, st>>>(ul, D.d_count, NSl, ul_names);
            LOR_LAUNCH_CHECK();
        }
        {
            ProfScope ps(PK_NAMING, double(hU) * (8 + 16 + 4), st);
            k_dbl_text_pairs<<<g, 256, 0, st>>>(ul, ul_names, int64_t(hU), SAR, Rl, r_unwritten ? headof : nullptr, T0->s,
                                                T0->n, T0->n0, T0->maxc, T0->kchars, runid);
            LOR_LAUNCH_CHECK();
        }
        {
            ProfScope ps(PK_NAMING, double(hU) * 8, st);
            const int64_t ntiles = cdiv(hU, kScanTile);
            LOR_TILE_LAUNCH(D, hU, k_dbl_keep, runid, ul, int64_t(hU), ul2, D.d_count, LB_ARGS(D), ntiles);
        }
        rc = read_u32(D, D.d_count, &hU);
        if (rc) return rc;
        uint32_t *t = ul;
        ul = ul2;
        ul2 = t;
    } else if (r_unwritten && hU > 0) {
        ProfScope ps(PK_NAMING, double(hU) * 24, st);
        const unsigned g = unsigned(min64(cdiv(hU, 256), 152 * 8));
        k_dbl_group_heads<<<g, 256, 0, st>>>(ul, D.d_count, NSl, headof);
        LOR_LAUNCH_CHECK();
        k_dbl_group_ranks<<<g, 256, 0, st>>>(ul, D.d_count, NSl, SAR, headof, Rl);
        LOR_LAUNCH_CHECK();
    }
    const int shift = bit_width_u64(uint64_t(m));
    for (int64_t h = 1; hU > 0; h *= 2) {
        if (h >= m) return LOR_ERR_BAD_INPUT;  // cannot happen for a valid R
        const int64_t U = hU;
        if (U <= kDblSmall) {
            ProfScope ps(PK_NAMING, double(U) * 48, st);
            const size_t smem = sizeof(DblSmallSmem);
            LOR_CUDA_TRY(cudaFuncSetAttribute(k_dbl_small, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_dbl_small<<<1, kDblSmallThreads, smem, st>>>(ul, D.d_count, m, h, shift, SAR, Rl, D.status, 0);
            LOR_LAUNCH_CHECK();
            break;
        }
        {
            ProfScope ps(PK_SAMPLE_KEYS, double(U) * 24, st);
            k_dbl_keys<<<grid_for(U, 256), 256, 0, st>>>(ul, U, SAR, Rl, m, h, shift, k0, val);
            LOR_LAUNCH_CHECK();
        }
        uint64_t *kr;
        uint32_t *vr;
        rc = radix_sort_pairs<uint64_t>(D.rs, k0, val, k1, valt, U, 0, 2 * shift, false, &kr, &vr);
        if (rc) return rc;
        {
            ProfScope ps(PK_NAMING, double(U) * 32, st);
            LOR_TILE_LAUNCH(D, U, k_dbl_runs, kr, vr, ul, U, SAR, runid, rstart, D.d_names, LB_ARGS(D));
            k_dbl_rank<<<grid_for(U, 256), 256, 0, st>>>(vr, runid, rstart, ul, U, Rl);
            LOR_LAUNCH_CHECK();
            const int64_t ntiles = cdiv(U, kScanTile);
            LOR_TILE_LAUNCH(D, U, k_dbl_next, runid, ul, U, ul2, D.d_count, LB_ARGS(D), ntiles);
        }
        rc = read_u32(D, D.d_count, &hU);
        if (rc) return rc;
        uint32_t *t = ul;
        ul = ul2;
        ul2 = t;
    }
    return LOR_OK;
}

// Step 2 by sorting: nonsample positions 3r for every B1 sample r in rank
// order, keyed by their first symbol, then one stable radix sort by it.
template <typename CharT>
int nonsample_by_sort(Dc3Run &D, const CharT *s, const LevelSizes &z, int bits, const int32_t *SAR,
                      const uint32_t **B) {
    cudaStream_t st = D.s;
    uint32_t *k0 = (uint32_t *)D.t64[1], *k1 = (uint32_t *)D.t64[2];
    {
        ProfScope ps(PK_NONSAMPLE, double(z.n02) * 4 + double(z.n0) * (sizeof(CharT) + 8), st);
        LOR_TILE_LAUNCH(D, z.n02, k_nonsample<CharT>, SAR, z.n02, z.n0, s, z.n, k0, D.t32[4], LB_ARGS(D));
    }
    uint32_t *kr, *vr;
    const int rc = radix_sort_pairs<uint32_t>(D.rs, k0, D.t32[4], k1, D.t32[5], z.n0, 0, bits, false, &kr, &vr);
    if (rc) return rc;
    *B = vr;
    return LOR_OK;
}

// Step 3: merge of the sample order (SAR, ranks in Rl) and the nonsample
// order B into out (the dummy, when present, is the smallest sample).  The
// records go to the two adjacent 64-bit buffers.
template <typename CharT>
int merge_run(Dc3Run &D, const LevelSizes &z, const GroupRec<CharT> *rec, const int32_t *SAR, const uint32_t *B,
              const BRec16 *Bx, const uint64_t *Ax, int32_t *out);

// The group records of Step 3 (rank(S_x) from Rl) in t64[1..2].
template <typename CharT>
int build_records(Dc3Run &D, const CharT *s, const LevelSizes &z, const int32_t *Rl, GroupRec<CharT> **rec_out) {
    cudaStream_t st = D.s;
    GroupRec<CharT> *rec = (GroupRec<CharT> *)D.t64[1];
    const size_t rec_bytes = align256(sizeof(GroupRec<CharT>) * size_t(z.n0));
    // The records fill at most t64[1..2] (16 bytes per position at level 0,
    // 32 per group of three below).
    if (rec_bytes > size_t((char *)D.t64[2] - (char *)D.t64[1]) * 2) return LOR_ERR_WORKSPACE;
    {
        ProfScope ps(PK_MERGE, double(z.n0) * (3.0 * sizeof(CharT) + 12 + sizeof(GroupRec<CharT>)), st);
        k_group_records<CharT><<<grid_for(z.n0, 256), 256, 0, st>>>(s, z.n, z.n0, z.n2, Rl, rec);
    }
    LOR_LAUNCH_CHECK();
    *rec_out = rec;
    return LOR_OK;
}

// Steps 2 and 3 at level 0.  Every sample's merge key goes to Ax in sample
// order by a bucketed scatter keyed by its rank (the keys are made from the
// text and the ranks read in sequence, and the scatter writes into
// L2-sized windows), so no step reads a record at random; the nonsample split
// then reads SAR and Ax in sequence (into t32[0..3]), and the merge reads
// both orders in sequence.
int level0_nonsample_and_merge(Dc3Run &D, const uint8_t *s, const LevelSizes &z, int64_t maxc, const int32_t *Rl,
                               const int32_t *SAR, int32_t *out) {
    const bool small_codes = maxc < 16;  // the split ranks 4-bit symbols
    cudaStream_t st = D.s;
    BRec16 *Bx = (BRec16 *)D.t32[0];
    if (size_t((char *)D.t32[4] - (char *)D.t32[0]) < sizeof(BRec16) * size_t(z.n0)) return LOR_ERR_WORKSPACE;
    uint64_t *Ax = D.t64[0];  // 8 bytes per sample, in sample order
    const int64_t m = z.n02;
    {
        // (j, key) pairs bucketed by the top 8 bits of j: a permutation of
        // [0, m), so every bucket's size is known without counting
        uint32_t *kb = D.t32[4];
        uint64_t *vb = D.t64[1];
        const int top = bit_width_u64(uint64_t(m > 1 ? m - 1 : 1));
        const int lo = top > kRadixBits ? top - kRadixBits : 0;
        k_perm_offsets<<<1, kRadix, 0, st>>>(D.rs.offsets, lo, m);
        LOR_LAUNCH_CHECK();
        {
            ProfScope ps(PK_NONSAMPLE, double(m) * (8 + 4.0 / 3.0 + 4 + 8), st);
            const int rc = launch_partition<uint32_t, uint64_t>(SampleKeySrc{s, Rl, z.n, z.n0, z.n2}, kb, vb, m,
                                                                nullptr, lo, digit_mask(lo, top), D.rs.offsets,
                                                                D.status, st);
            if (rc) return rc;
        }
        LOR_LAUNCH_CHECK();
        {
            ProfScope ps(PK_NONSAMPLE, double(m) * (4 + 8 + 8), st);
            k_scatter_u64<<<grid_for(m, 256), 256, 0, st>>>(kb, vb, m, Ax, m, D.status);
        }
        LOR_LAUNCH_CHECK();
    }
    LOR_CUDA_TRY(cudaMemsetAsync(D.rs.hist, 0, sizeof(uint32_t) * kRadix, st));
    {
        ProfScope ps(PK_NONSAMPLE, double(z.n0), st);
        k_first_sym_hist<<<unsigned(min64(cdiv(z.n0, 256), 152 * 4)), 256, 0, st>>>(s, z.n0, D.rs.hist);
        LOR_LAUNCH_CHECK();
        k_radix_offsets<<<1, kRadix, 0, st>>>(D.rs.hist, D.rs.offsets);
        LOR_LAUNCH_CHECK();
    }
    {
        const int64_t ntiles = cdiv(m, kSpTile);
        const int64_t per = cdiv(ntiles, kSpRanges);
        const int nranges = int(cdiv(ntiles, per));
        uint32_t *cnt = (uint32_t *)(D.ws + D.L.ns_table);
        uint32_t *part = cnt + ntiles * kRadix;
        if (ntiles > cdiv(D.L.max_m, kSpTile)) return LOR_ERR_WORKSPACE;
        // resident grids: four count blocks, three write blocks per SM
        const unsigned grid = unsigned(min64(ntiles, int64_t(sort_grid_cap())));
        const unsigned wgrid = unsigned(min64(ntiles, int64_t(sort_grid_cap()) / 4 * 3));
        {
            ProfScope ps(PK_NONSAMPLE, double(m) * 8, st);
            auto kern = small_codes ? k_ns_count<4> : k_ns_count<8>;
            LOR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(sizeof(NsCountSmem))));
            kern<<<grid, kSortThreads, sizeof(NsCountSmem), st>>>(Ax, m, cnt, D.status);
            LOR_LAUNCH_CHECK();
        }
        {
            ProfScope ps(PK_NONSAMPLE, double(ntiles) * kRadix * 12, st);
            k_ns_scan_ranges<<<unsigned(nranges), kRadix, 0, st>>>(cnt, ntiles, per, part);
            LOR_LAUNCH_CHECK();
            k_ns_scan_starts<<<1, kRadix, 0, st>>>(part, nranges, D.rs.offsets);
            LOR_LAUNCH_CHECK();
            k_ns_scan_tiles<<<unsigned(nranges), kRadix, 0, st>>>(cnt, ntiles, per, part);
            LOR_LAUNCH_CHECK();
        }
        {
            ProfScope ps(PK_NONSAMPLE, double(m) * 4 + double(z.n0) * (8 + 16), st);
            auto kern = small_codes ? k_ns_write<4> : k_ns_write<8>;
            LOR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(sizeof(NsWriteSmem))));
            kern<<<wgrid, kSortThreads, sizeof(NsWriteSmem), st>>>(SAR, Ax, m, z.n0, cnt, Bx, D.status);
            LOR_LAUNCH_CHECK();
        }
    }
    return merge_run<uint8_t>(D, z, nullptr, SAR, nullptr, Bx, Ax, out);
}

template <typename CharT>
int merge_level(Dc3Run &D, const CharT *s, const LevelSizes &z, const int32_t *Rl, const int32_t *SAR,
                const uint32_t *B, int32_t *out) {
    GroupRec<CharT> *rec;
    const int rc = build_records<CharT>(D, s, z, Rl, &rec);
    if (rc) return rc;
    return merge_run<CharT>(D, z, rec, SAR, B, nullptr, nullptr, out);
}

template <typename CharT>
int merge_run(Dc3Run &D, const LevelSizes &z, const GroupRec<CharT> *rec, const int32_t *SAR, const uint32_t *B,
              const BRec16 *Bx, const uint64_t *Ax, int32_t *out) {
    cudaStream_t st = D.s;
    const int64_t n = z.n;
    MergeIn<CharT> a;
    a.rec = rec;
    a.n0 = int32_t(z.n0);
    const int64_t dummy = (z.n0 > z.n1) ? 1 : 0;
    a.A = SAR + dummy;
    a.na = z.n02 - dummy;
    a.B = B;
    a.nb = z.n0;
    a.Bx = Bx;
    a.Ax = Ax ? Ax + dummy : nullptr;
    const int64_t ntiles = cdiv(n, kMergeTile);
    int64_t *split = (int64_t *)(D.ws + D.L.split);
    {
        ProfScope ps(PK_MERGE, double(n) * (4 + 4 + sizeof(GroupRec<CharT>)), st);
        k_merge_partition<CharT><<<grid_for(ntiles + 1, 128), 128, 0, st>>>(a, ntiles, split);
        LOR_LAUNCH_CHECK();
        const int mi = tune_config().merge_items;
        if constexpr (sizeof(CharT) == 1) {
            if (Ax && Bx) {
                if (mi == 8)
                    k_merge_packed<8><<<unsigned(ntiles), kMergeTile / 8, 0, st>>>(a, split, out, D.status);
                else if (mi == 4)
                    k_merge_packed<4><<<unsigned(ntiles), kMergeTile / 4, 0, st>>>(a, split, out, D.status);
                else
                    k_merge_packed<2><<<unsigned(ntiles), kMergeTile / 2, 0, st>>>(a, split, out, D.status);
                LOR_LAUNCH_CHECK();
                return LOR_OK;
            }
        }
        if (mi == 8)
            k_merge<CharT, 8><<<unsigned(ntiles), kMergeTile / 8, 0, st>>>(a, split, out, D.status);
        else if (mi == 4)
            k_merge<CharT, 4><<<unsigned(ntiles), kMergeTile / 4, 0, st>>>(a, split, out, D.status);
        else
            k_merge<CharT, 2><<<unsigned(ntiles), kMergeTile / 2, 0, st>>>(a, split, out, D.status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}


// Doubling replaces the next level when at most 1/kDoublingShare of the
// samples lost their name to a duplicate (lor_dc3_route_set's doubling
// route: 0 never, 2 whenever names repeat).
constexpr int64_t kDoublingShare = 16;

// ---- prefix doubling with every round enqueued up front (graph mode)
//
// The unresolved count stays on the device: round r (step h = 2^r) reads it,
// and its kernels do nothing once it is 0.  bit_width(m) rounds always
// finish (after the round with step h the order is by 2h symbols of R, and
// 2h >= m suffices); the single-block tail runs after the second round and
// again after the last, taking over whenever few samples are left.
int sa_by_doubling_graph(Dc3Run &D, int32_t *Rl, int64_t m, int32_t *SAR, const int32_t *NSl,
                         bool r_unwritten) {
    cudaStream_t st = D.s;
    int32_t *headof = (int32_t *)D.t32[0];
    uint32_t *ul = D.t32[1], *ul2 = D.t32[2], *runid = D.t32[3], *val = D.t32[4], *rstart = D.t32[5];
    uint32_t *valt = D.t32[0];
    uint64_t *k0 = D.t64[0], *k1 = D.t64[1];
    uint32_t *cnt = D.d_count, *cnt2 = D.d_count + 1;
    if (r_unwritten) {
        int rc = bucketed_scatter(D.rs, (const uint32_t *)SAR, nullptr, m, m, D.t32[2], D.t32[3], D.t32[4], Rl, 1);
        if (rc) return rc;
    } else {
        k_dbl_headof<<<grid_for(m, 256), 256, 0, st>>>(NSl, m, headof);
        LOR_LAUNCH_CHECK();
        k_dbl_init<<<grid_for(m, 256), 256, 0, st>>>(Rl, m, headof);
        LOR_LAUNCH_CHECK();
    }
    {
        const int64_t ntiles = cdiv(m, kScanTile);
        LOR_PTILE_LAUNCH(D, m, k_dbl_unresolved, NSl, m, ul, cnt, LB_ARGS(D), ntiles);
    }
    if (r_unwritten) {
        const unsigned g = unsigned(min64(cdiv(m, 256), scan_grid_cap()));
        k_dbl_group_heads<<<g, 256, 0, st>>>(ul, cnt, NSl, headof);
        LOR_LAUNCH_CHECK();
        k_dbl_group_ranks<<<g, 256, 0, st>>>(ul, cnt, NSl, SAR, headof, Rl);
        LOR_LAUNCH_CHECK();
    }
    const int shift = bit_width_u64(uint64_t(m));
    const int rounds = shift > 0 ? shift : 1;
    const size_t small_smem = sizeof(DblSmallSmem);
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_dbl_small, cudaFuncAttributeMaxDynamicSharedMemorySize, int(small_smem)));
    const unsigned gcap = scan_grid_cap();
    const unsigned ggrid = unsigned(min64(cdiv(m, 256), gcap));
    for (int r = 0; r < rounds; ++r) {
        const int64_t h = int64_t(1) << r;
        k_dbl_keys_dev<<<ggrid, 256, 0, st>>>(ul, cnt, SAR, Rl, m, h, shift, k0, val);
        LOR_LAUNCH_CHECK();
        uint64_t *kr;
        uint32_t *vr;
        int rc = radix_sort_pairs<uint64_t>(D.rs, k0, val, k1, valt, m, 0, 2 * shift, false, &kr, &vr, false, cnt);
        if (rc) return rc;
        unsigned long long *ctr, base;
        rc = take_counter(D.rs, true, &ctr, &base);
        if (rc) return rc;
        D.rs.epoch++;
        k_dbl_runs_dev<<<unsigned(min64(cdiv(m, kScanTile), gcap)), kScanThreads, 0, st>>>(
            kr, vr, ul, cnt, SAR, runid, rstart, D.rs.lookback, ctr, D.rs.epoch, D.status);
        LOR_LAUNCH_CHECK();
        k_dbl_rank_dev<<<ggrid, 256, 0, st>>>(vr, runid, rstart, ul, cnt, Rl);
        LOR_LAUNCH_CHECK();
        rc = take_counter(D.rs, true, &ctr, &base);
        if (rc) return rc;
        D.rs.epoch++;
        k_dbl_next_dev<<<unsigned(min64(cdiv(m, kScanTile), gcap)), kScanThreads, 0, st>>>(
            runid, ul, cnt, ul2, cnt2, D.rs.lookback, ctr, D.rs.epoch, D.status);
        LOR_LAUNCH_CHECK();
        uint32_t *t = ul;
        ul = ul2;
        ul2 = t;
        t = cnt;
        cnt = cnt2;
        cnt2 = t;
        if (r == 1 || r == rounds - 1) {
            k_dbl_small<<<1, kDblSmallThreads, small_smem, st>>>(ul, cnt, m, 2 * h, shift, SAR, Rl, D.status, 1);
            LOR_LAUNCH_CHECK();
        }
    }
    k_dbl_check_done<<<1, 32, 0, st>>>(cnt, D.status);
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

// DC3 with no host round trip, for capture in a CUDA graph: level 0 sorts
// its sample by the 48-bit prefix, its reduced string is finished by the
// enqueued doubling rounds above (whatever the number of repeated names),
// then Steps 2 and 3 as in dc3_level.
int dc3_graph(Dc3Run &D, const uint8_t *s, int64_t n, int64_t maxc, int32_t *out) {
    cudaStream_t st = D.s;
    const LevelSizes z = level_sizes(n);
    int32_t *Rl = (int32_t *)(D.ws + D.L.lev_R[0]);
    int32_t *SAR = (int32_t *)(D.ws + D.L.lev_SAR[0]);
    int32_t *NSl = (int32_t *)(D.ws + D.L.lev_NS[0]);
    const int bits = bit_width_u64(uint64_t(maxc));
    const int kchars = level0_kchars(bits, maxc);
    uint64_t T = 1;
    for (int t = 0; t < kchars && T; ++t)
        T = T > ~uint64_t(0) / (uint64_t(maxc) + 1) ? 0 : T * (uint64_t(maxc) + 1);
    if (!T) return LOR_ERR_INVALID_ARG;
    const int key_bits = bit_width_u64(T - 1);
    LOR_CUDA_TRY(cudaMemsetAsync(Rl + z.n02, 0, sizeof(int32_t) * kPad, st));
    int rc = key_bits <= 32
                 ? sample_sort_and_name<uint8_t, uint32_t>(D, 0, s, z, kchars, key_bits, maxc, Rl, SAR, NSl)
                 : sample_sort_and_name<uint8_t, uint64_t>(D, 0, s, z, kchars, key_bits, maxc, Rl, SAR, NSl);
    if (rc) return rc;
    rc = sa_by_doubling_graph(D, Rl, z.n02, SAR, NSl, bucket_names(D, z));
    if (rc) return rc;
    return level0_nonsample_and_merge(D, s, z, maxc, Rl, SAR, out);
}

template <typename CharT>
int dc3_level(Dc3Run &D, int lvl, const CharT *s, int64_t n, int64_t maxc, int32_t *out, const int32_t *PS,
              const int32_t *PNS) {
    cudaStream_t st = D.s;
    if (lvl >= int(D.L.lev_R.size())) return LOR_ERR_WORKSPACE;
    const LevelSizes z = level_sizes(n);
    int32_t *Rl = (int32_t *)(D.ws + D.L.lev_R[lvl]);
    int32_t *SAR = (int32_t *)(D.ws + D.L.lev_SAR[lvl]);
    int32_t *NSl = (int32_t *)(D.ws + D.L.lev_NS[lvl]);
    const int bits = bit_width_u64(uint64_t(maxc));
    const int kchars = lvl == 0 ? level0_kchars(bits, maxc) : 3;
    // Keys are the kchars symbols as digits of base maxc + 1 (most significant
    // first): T = (maxc + 1)^kchars distinct keys, 0 when that overflows 64 bits.
    uint64_t T = 1;
    for (int t = 0; t < kchars && T; ++t)
        T = T > ~uint64_t(0) / (uint64_t(maxc) + 1) ? 0 : T * (uint64_t(maxc) + 1);
    int key_bits = T ? bit_width_u64(T - 1) : kchars * bits;

    LOR_CUDA_TRY(cudaMemsetAsync(Rl + z.n02, 0, sizeof(int32_t) * kPad, st));
    int rc;
    uint32_t names = 0;
    int strategy;
    int64_t dups = 0;
    bool sorted_list = true;  // SAR / NSl hold the samples in key order
    bool packed = false;
    if constexpr (sizeof(CharT) == 1) {
        if (lvl == 0 && g_route_k0.load(std::memory_order_relaxed) == 0) {
            rc = sample_packed_sort_and_name(D, s, z, maxc, Rl, SAR, NSl, &packed);
            if (rc) return rc;
        }
    }
    if (packed) {
        strategy = 0;
        key_bits = 33;
        rc = read_u32(D, D.d_names, &names);
    } else if (PS && !D.force_lsd) {
        strategy = 2;
        rc = sample_from_parent<CharT>(D, s, z, bits, PS, PNS, Rl, SAR, NSl, &dups);
        if (rc) return rc;
        rc = read_u32(D, D.d_names, &names);
    } else if (!D.force_lsd && T && T <= uint64_t(D.L.tbl_entries)) {
        strategy = 1;
        rc = sample_dense_names<CharT>(D, lvl, s, z, kchars, int64_t(T), maxc, Rl, SAR, NSl, &names);
        sorted_list = int64_t(names) == z.n02;
    } else {
        strategy = 0;
        if (T && key_bits <= 32)
            rc = sample_sort_and_name<CharT, uint32_t>(D, lvl, s, z, kchars, key_bits, maxc, Rl, SAR, NSl);
        else if (T)
            rc = sample_sort_and_name<CharT, uint64_t>(D, lvl, s, z, kchars, key_bits, maxc, Rl, SAR, NSl);
        else rc = sample_sort_and_name_wide<CharT>(D, s, z, bits, maxc, Rl, SAR, NSl);
        if (rc) return rc;
        rc = read_u32(D, D.d_names, &names);
    }
    if (rc) return rc;
    g_trace.push_back(TraceRow{n, int64_t(names), key_bits});
    g_trace_extra.push_back(TraceExtra{strategy, dups});
    const int64_t lost = z.n02 - int64_t(names);
    const bool doubling = lost > 0 && sorted_list &&
                          (D.doubling == 2 || (D.doubling == 1 && lost * kDoublingShare <= z.n02));
    // Sorted large levels left R unwritten; doubling writes ranks there itself.
    const bool r_unwritten = strategy != 1 && bucket_names(D, z);
    if (r_unwritten && !doubling) {
        rc = names_scatter(D, SAR, NSl, z.n02, Rl);
        if (rc) return rc;
    }
    if (doubling) {
        int64_t u0 = 0;
        Level0Text T0;
        if constexpr (sizeof(CharT) == 1) {
            if (lvl == 0) {
                T0.s = s;
                T0.n = z.n;
                T0.n0 = z.n0;
                T0.maxc = uint32_t(maxc);
                T0.kchars = packed ? kPkChars : kchars;
            }
        }
        rc = sa_by_doubling(D, Rl, z.n02, SAR, NSl, r_unwritten, &u0, packed, T0.s ? &T0 : nullptr);
        if (rc) return rc;
        g_trace.push_back(TraceRow{z.n02, z.n02, 0});
        g_trace_extra.push_back(TraceExtra{3, u0});
    } else if (lost > 0) {
        rc = dc3_level<int32_t>(D, lvl + 1, Rl, z.n02, int64_t(names), SAR, sorted_list ? SAR : nullptr,
                                sorted_list ? NSl : nullptr);
        if (rc) return rc;
        rc = rank_scatter(D, SAR, z.n02, Rl);
        if (rc) return rc;
    }
    // Rl now holds rank(S_i) by reduced-string index (unique names are ranks).

    // Step 2: nonsample order, as group indices t (position 3t).
    if constexpr (sizeof(CharT) == 1) {
        if (!PS && !D.force_lsd) return level0_nonsample_and_merge(D, s, z, maxc, Rl, SAR, out);
    }
    const uint32_t *B;
    if (PS && !D.force_lsd) {
        uint32_t *T0 = D.t32[0], *P0 = D.t32[1], *Dslot = D.t32[2], *Dt = D.t32[3];
        uint32_t *Dkey = (uint32_t *)D.t64[1];
        {
            ProfScope ps(PK_NONSAMPLE, double(n) * 8 + double(z.n0) * 8, st);
            LOR_TILE_LAUNCH(D, n, k_par_nonsamples, PS, PNS, n, T0, P0, LB_ARGS(D));
        }
        {
            ProfScope ps(PK_NONSAMPLE, double(z.n0) * 4, st);
            const int64_t ntiles = cdiv(z.n0, kScanTile);
            LOR_TILE_LAUNCH(D, z.n0, k_par_ns_dups, T0, P0, z.n0, Rl, Dslot, Dt, Dkey, D.d_count, LB_ARGS(D),
                            ntiles);
        }
        uint32_t nd = 0;
        rc = read_u32(D, D.d_count, &nd);
        if (rc) return rc;
        if (nd > 0) {
            uint32_t *vord;
            const int rank_bits = bit_width_u64(uint64_t(z.n02));
            rc = sort_dups_then_by_first<uint32_t>(D, Dkey, nd, rank_bits, Dslot, P0, bits, &vord);
            if (rc) return rc;
            k_par_ns_writeback<<<grid_for(nd, 256), 256, 0, st>>>(vord, nd, Dslot, Dt, T0);
            LOR_LAUNCH_CHECK();
        }
        B = T0;
    } else {
        rc = nonsample_by_sort<CharT>(D, s, z, bits, SAR, &B);
        if (rc) return rc;
    }

    return merge_level<CharT>(D, s, z, Rl, SAR, B, out);
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_build_sa_workspace_size(int64_t n, int32_t sigma) {
    (void)sigma;
    if (n < 1 || n > LOR_MAX_N) return 0;
    return dc3_layout(n).total;
}

extern "C" int lor_build_sa(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa, void *d_ws,
                            size_t ws_bytes, lor_stream_t stream) {
    return lor::build_sa_impl(d_text, n, sigma, d_sa, d_ws, ws_bytes, (cudaStream_t)stream, nullptr, 0);
}

int lor::build_sa_impl(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa, void *d_ws,
                       size_t ws_bytes, cudaStream_t stream, unsigned long long *graph_ctr_pool,
                       int graph_pool_size) {
    if (!d_text || !d_sa || n < 1 || sigma < 2 || sigma > 256) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const bool graph = graph_ctr_pool != nullptr;
    Dc3Run D;
    D.L = dc3_layout(n);
    if (!d_ws || ws_bytes < D.L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    D.s = (cudaStream_t)stream;
    D.status = tu_status_ptr();
    if (!D.status) return LOR_ERR_CUDA;
    D.ws = (char *)d_ws;
    D.d_names = (uint32_t *)(D.ws + D.L.ctrl);
    D.rs.hist = (uint32_t *)(D.ws + D.L.hist);
    D.rs.offsets = (uint32_t *)(D.ws + D.L.offsets);
    D.rs.lookback = (uint64_t *)(D.ws + D.L.lookback);
    D.rs.tile_ctr = (unsigned long long *)(D.ws + D.L.ctrl + 64);
    D.rs.max_tiles = cdiv(D.L.max_m, kMinSortTile);
    D.rs.status = D.status;
    D.rs.stream = D.s;
    for (int i = 0; i < 3; ++i) D.t64[i] = (uint64_t *)(D.ws + D.L.t64[i]);
    for (int i = 0; i < 6; ++i) D.t32[i] = (uint32_t *)(D.ws + D.L.t32[i]);
    D.tbl = (uint32_t *)(D.ws + D.L.tbl);
    D.d_count = (uint32_t *)(D.ws + D.L.ctrl + 128);
    D.force_lsd = g_route_strategy.load(std::memory_order_relaxed) == 1;  // radix-sort every level
    D.doubling = g_route_doubling.load(std::memory_order_relaxed);
    LOR_CUDA_TRY(cudaMemsetAsync(D.ws + D.L.ctrl, 0, 256, D.s));
    LOR_CUDA_TRY(cudaMemsetAsync(D.ws + D.L.lookback, 0, D.L.lookback_bytes, D.s));
    g_trace.clear();
    g_trace_extra.clear();
    if (graph) {
        D.rs.graph = true;
        D.rs.ctr_pool = graph_ctr_pool;
        D.rs.ctr_pool_size = graph_pool_size;
        LOR_CUDA_TRY(cudaMemsetAsync(graph_ctr_pool, 0, sizeof(unsigned long long) * size_t(graph_pool_size), D.s));
        D.force_lsd = false;
        return dc3_graph(D, d_text, n, int64_t(sigma - 1), d_sa);
    }
    return dc3_level<uint8_t>(D, 0, d_text, n, int64_t(sigma - 1), d_sa, nullptr, nullptr);
}

extern "C" int lor_dc3_route_set(int32_t level0_symbols, int32_t strategy, int32_t doubling) {
    if (level0_symbols < 0 || level0_symbols > kKeyMaxChars || level0_symbols == 2 ||
        strategy < 0 || strategy > 1 || doubling < 0 || doubling > 2)
        return LOR_ERR_INVALID_ARG;
    g_route_k0.store(level0_symbols);
    g_route_strategy.store(strategy);
    g_route_doubling.store(doubling);
    return LOR_OK;
}

extern "C" int lor_dc3_route_get(int32_t *level0_symbols, int32_t *strategy, int32_t *doubling) {
    if (level0_symbols) *level0_symbols = g_route_k0.load();
    if (strategy) *strategy = g_route_strategy.load();
    if (doubling) *doubling = g_route_doubling.load();
    return LOR_OK;
}

extern "C" int lor_last_dc3_trace(int64_t *h_n, int64_t *h_names, int32_t *h_key_bits,
                                  int32_t *h_strategy, int64_t *h_dups, int32_t cap) {
    const int cnt = int(g_trace.size());
    for (int i = 0; i < cnt && i < cap; ++i) {
        if (h_n) h_n[i] = g_trace[i].n;
        if (h_names) h_names[i] = g_trace[i].names;
        if (h_key_bits) h_key_bits[i] = g_trace[i].key_bits;
        if (h_strategy) h_strategy[i] = g_trace_extra[i].strategy;
        if (h_dups) h_dups[i] = g_trace_extra[i].dups;
    }
    return cnt;
}
