// radix.cuh -- stable LSD radix sort of (key, uint32 value) pairs.
//
// The paper's DC3 sorts its sample triples and nonsample pairs with an LSD
// radix sort (Section 4, Algorithm 1: one 1-bit split per pass, block-local
// chunks merged afterwards).  Here one pass moves 8 bits: an up-front
// histogram kernel counts every pass's digits in one read of the keys, and
// each pass is a single "onesweep" kernel -- a block counts its tile's digits
// and publishes them for the tiles after it, ranks the keys stably with warp
// ballots, learns the global offset of each digit from its predecessors by
// decoupled look-back (bounded waits), and scatters through shared memory so
// that every digit run is written contiguously.
#pragma once

#include <cstdlib>

#include "common.cuh"

namespace lor {

constexpr int kRadixBits = 8;
constexpr int kRadix = 256;
constexpr int kSortThreads = 256;  // == kRadix: one thread per digit in the look-back
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxPasses = 16;  // 64-bit keys at 4-bit digits

// Keys per thread: sized so that four 256-thread blocks fit an SM (64
// registers per thread, under 57 KB of shared memory per block; the few
// spilled registers cost less than the occupancy they buy).
template <typename KeyT, typename ValT = uint32_t>
__host__ __device__ constexpr int sort_items() { return sizeof(KeyT) + sizeof(ValT) > 8 ? 12 : 16; }
template <typename KeyT, typename ValT = uint32_t>
__host__ __device__ constexpr int sort_tile() { return kSortThreads * sort_items<KeyT, ValT>(); }

// Where a pass takes its values from.
enum ValMode {
    VM_LOAD = 0,      // vin[idx]
    VM_IOTA = 1,      // idx (32-bit values)
    VM_IDX_PREV = 2,  // 64-bit values: low word idx, high word the previous key (kin[idx-1], or ~0)
};
constexpr int kMinSortTile = kSortThreads * 8;  // the smallest tile of any pass

// Lanes of the warp holding the same 9-bit value d as this lane (digit, or
// 0x100 for an empty slot): one ballot per bit, kept or inverted by this
// lane's bit.  The same set as __match_any_sync, from cheap vote instructions.
__device__ __forceinline__ uint32_t warp_peers9(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// The same for an N-bit value.
template <int N>
__device__ __forceinline__ uint32_t warp_peers_bits(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < N; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// The same for an 8-bit value (every slot valid).
__device__ __forceinline__ uint32_t warp_peers8(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift, uint32_t mask = 0xFFu) {
    return uint32_t(k >> shift) & mask;
}
// Digit mask of the pass starting at `shift` when the key ends at end_bit
// (digits of `bits` bits, at most 8).
__host__ __device__ __forceinline__ uint32_t digit_mask(int shift, int end_bit, int bits = kRadixBits) {
    const int w = end_bit - shift < bits ? end_bit - shift : bits;
    return (1u << w) - 1u;
}

// Digit histograms of every pass in one read of the keys.  Counts go to
// shared-memory atomics; when all 32 lanes of a warp hold the same digit (low
// entropy passes) one lane adds 32 instead.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_radix_hist(const KeyT *__restrict__ keys, int64_t m,
                                                    const uint32_t *m_dev, int begin_bit, int end_bit,
                                                    int npasses, int dbits, uint32_t *__restrict__ hist) {
    if (m_dev) m = int64_t(*m_dev);
    __shared__ uint32_t sh[kMaxPasses * kRadix];
    for (int i = threadIdx.x; i < npasses * kRadix; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    constexpr int kPer = 4;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * kPer;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x * kPer; base < m; base += stride) {
        KeyT k[kPer];
        bool valid[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int64_t i = base + u * int64_t(blockDim.x) + threadIdx.x;
            valid[u] = i < m;
            k[u] = valid[u] ? keys[i] : KeyT(0);
        }
        for (int p = 0; p < npasses; ++p) {
            const int sft = begin_bit + p * dbits;
            const uint32_t dm = digit_mask(sft, end_bit, dbits);
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint32_t d = digit_of(k[u], sft, dm);
                const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
                const bool all_valid = __all_sync(0xffffffffu, valid[u]);
                if (all_valid && __all_sync(0xffffffffu, d == d0)) {
                    if (lane == 0) atomicAdd(&sh[p * kRadix + d0], 32u);
                } else if (valid[u]) {
                    atomicAdd(&sh[p * kRadix + d], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npasses * kRadix; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each pass's 256 digit counts (one block per pass).
static __global__ void __launch_bounds__(256) k_radix_offsets(const uint32_t *__restrict__ hist,
                                                       uint32_t *__restrict__ offsets) {
    __shared__ uint32_t scratch[kRadix / 32 + 1];
    const int p = blockIdx.x;
    uint32_t total;
    const uint32_t v = hist[p * kRadix + threadIdx.x];
    offsets[p * kRadix + threadIdx.x] = block_excl_scan<kRadix>(v, scratch, &total);
}

template <typename KeyT, typename ValT, int kItems = sort_items<KeyT, ValT>()>
struct OnesweepSmem {
    KeyT keys[kSortThreads * kItems];
    ValT vals[kSortThreads * kItems];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t early[kRadix];
    uint32_t local_start[kRadix];
    long long gbase[kRadix];
    uint32_t scratch[kSortWarps + 1];
    long long tile;
    long long next;
};

// Exclusive prefix of digit dg over the tiles before `tile`: walks back over
// the predecessors' descriptors, kLookWindow of them per round of independent
// loads (the walk is a chain of L2 round trips, so fewer rounds is less
// waiting), summing aggregates up to the first inclusive prefix.  A
// descriptor not yet published ends the round; the walk resumes there.  The
// whole wait is bounded by the wait limit (then LOR_ERR_TIMEOUT).
constexpr int kLookWindow = 2;

__device__ __forceinline__ uint32_t lookback_digit(const uint64_t *lb, int64_t tile, int dg, uint32_t epoch,
                                                   int *status) {
    uint32_t excl = 0;
    int64_t j = tile - 1;
    const uint64_t t0 = global_ns(), limit = wait_limit_ns();
    while (j >= 0) {
        uint64_t w[kLookWindow];
#pragma unroll
        for (int u = 0; u < kLookWindow; ++u)
            w[u] = j - u >= 0 ? ld_volatile_u64(&lb[(j - u) * kRadix + dg]) : lb_pack(epoch, kFlagIncl, 0);
        bool done = false;
        int used = 0;
#pragma unroll
        for (int u = 0; u < kLookWindow; ++u) {
            if (done || used < u) break;  // stop at the first descriptor not yet published
            if (lb_epoch(w[u]) != epoch || lb_flag(w[u]) == 0) break;
            excl += lb_value(w[u]);
            used = u + 1;
            if (lb_flag(w[u]) == kFlagIncl) done = true;
        }
        if (done) break;
        j -= used;
        if (used == 0 && global_ns() - t0 > limit) {
            atomicCAS(status, 0, LOR_ERR_TIMEOUT);
            break;
        }
    }
    return excl;
}

// One LSD pass over digit (shift .. shift+7).  A grid of a few blocks per SM
// stays resident and every block claims tiles from the running counter until
// it draws one past the end, so a tile only ever waits on tiles claimed
// before it by running blocks; each wait is still bounded by the wait limit.
// Every block makes exactly one claim past the last tile: a launch advances
// the counter by ntiles + gridDim.x.  When m_dev is given the element count
// is read from device memory (the count of an earlier kernel), so that the
// launch needs no host round trip.
// Four blocks per SM at 64 registers a thread; the widest tile of 64-bit keys
// (16 a thread) takes three blocks with more registers instead of spilling.
template <typename KeyT, int kItems>
__host__ __device__ constexpr int onesweep_min_blocks() { return sizeof(KeyT) == 8 && kItems > 12 ? 3 : 4; }

template <typename KeyT, typename ValT, int kVMode, int kItems>
__global__ void __launch_bounds__(kSortThreads, onesweep_min_blocks<KeyT, kItems>()) k_onesweep(
    const KeyT *__restrict__ kin, const ValT *__restrict__ vin, KeyT *__restrict__ kout,
    ValT *__restrict__ vout, int64_t m, const uint32_t *m_dev, int shift, uint32_t dmask,
    const uint32_t *__restrict__ offsets,
    uint64_t *__restrict__ lookback, unsigned long long *tile_ctr, unsigned long long tile_base,
    uint32_t epoch, int *status, int64_t ahead) {
    constexpr int kTile = kSortThreads * kItems;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<KeyT, ValT, kItems> &S = *reinterpret_cast<OnesweepSmem<KeyT, ValT, kItems> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (m_dev) m = int64_t(*m_dev);
    const int64_t ntiles = cdiv(m, kTile);
    const bool starve = g_starve_first_tile != 0;  // test switch, off in normal use
    // A claim also asks the L2 for the data of the tile `ahead` claims later.
    // (A tile is claimed only when its block is ready to work on it: a tile
    // claimed early would hold up the look-back of every later tile.)
    auto claim = [&]() {
        const long long t = (long long)(atomicAdd(tile_ctr, 1ull) - tile_base);
        const int64_t b2 = (t + ahead) * kTile;
        if (ahead > 0 && b2 < m) {
            const int64_t c2 = min64(int64_t(kTile), m - b2);
            const uint32_t kb = uint32_t(c2 * int64_t(sizeof(KeyT))) & ~15u;
            if (kb) prefetch_l2_bulk(kin + b2, kb);
            if (kVMode == VM_LOAD) {
                const uint32_t vb = uint32_t(c2 * int64_t(sizeof(ValT))) & ~15u;
                if (vb) prefetch_l2_bulk(vin + b2, vb);
            }
        }
        return t;
    };
    for (;;) {
        if (tid == 0) S.next = claim();
        for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&S.warp_hist[0][0])[i] = 0;
        S.early[tid] = 0;
        __syncthreads();
        const int64_t tile = S.next;
        if (tile >= ntiles) break;  // uniform over the block
        const int64_t base = tile * kTile;
        // positions inside the tile are 32-bit; the tile's pointers carry the base
        const int cnt_tile = int(min64(int64_t(kTile), m - base));
        const KeyT *kt = kin + base;
        const int wloc = warp * (kItems * 32) + lane;

        KeyT k[kItems];
        ValT v[kItems];
        uint32_t r[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int loc = wloc + i * 32;
            const bool valid = loc < cnt_tile;
            k[i] = valid ? kt[loc] : KeyT(0);
            if constexpr (kVMode == VM_LOAD) v[i] = valid ? vin[base + loc] : ValT(0);
            if constexpr (kVMode == VM_IDX_PREV)
                v[i] = uint64_t(uint32_t(base) + uint32_t(loc)) |
                       (uint64_t(valid && base + loc > 0 ? uint32_t(kt[loc - 1]) : 0xFFFFFFFFu) << 32);
        }
        // Early counts: the tile's digit totals from shared-memory atomics,
        // published before the (slower) stable ranking, so that later tiles'
        // look-back finds this tile's aggregate sooner.
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (wloc + i * 32 < cnt_tile) atomicAdd(&S.early[digit_of(k[i], shift, dmask)], 1u);
        __syncthreads();
        if (!(starve && tile == 0)) {
            const uint32_t e = S.early[tid];
            st_volatile_u64(&lookback[tile * kRadix + tid], lb_pack(epoch, tile == 0 ? kFlagIncl : kFlagAgg, e));
        }
        // Stable rank inside the warp: items in order, lanes in order.  The
        // lanes sharing each item's digit are found first for every item (the
        // ballots are independent of each other), then the warp's running
        // digit counts are walked item by item.  Slots past the end of the
        // input use digit 256 and are never counted (a whole tile has none,
        // and its ranking needs one ballot fewer).
        uint32_t *wh = S.warp_hist[warp];
        const uint32_t lt_mask = lanemask_lt();
        if (cnt_tile == kTile) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) r[i] = warp_peers8(digit_of(k[i], shift, dmask));
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const uint32_t d = digit_of(k[i], shift, dmask);
                const uint32_t peers = r[i];
                const uint32_t lt = __popc(peers & lt_mask);
                const uint32_t cnt = wh[d];
                r[i] = cnt + lt;
                __syncwarp();
                if (lt == 0) wh[d] = cnt + __popc(peers);
                __syncwarp();
            }
        } else {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const bool valid = wloc + i * 32 < cnt_tile;
                r[i] = warp_peers9(valid ? digit_of(k[i], shift, dmask) : 0x100u);
            }
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const bool valid = wloc + i * 32 < cnt_tile;
                const uint32_t d = valid ? digit_of(k[i], shift, dmask) : 0u;
                const uint32_t peers = r[i];
                const uint32_t lt = __popc(peers & lt_mask);
                const uint32_t cnt = valid ? wh[d] : 0u;
                r[i] = cnt + lt;
                __syncwarp();
                if (valid && lt == 0) wh[d] = cnt + __popc(peers);
                __syncwarp();
            }
        }
        __syncthreads();
        const int dg = tid;
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = S.warp_hist[w][dg];
            S.warp_hist[w][dg] = total;
            total += c;
        }
        uint32_t tile_total;
        const uint32_t lstart = block_excl_scan<kSortThreads>(total, S.scratch, &tile_total);
        S.local_start[dg] = lstart;

        // Decoupled look-back, one digit per thread (the aggregate, equal to
        // the early count, is already published).
        uint32_t excl = 0;
        uint64_t *lb = lookback;
        if (tile != 0) {
            excl = lookback_digit(lb, tile, dg, epoch, status);
            st_volatile_u64(&lb[tile * kRadix + dg], lb_pack(epoch, kFlagIncl, excl + total));
        }
        S.gbase[dg] = (long long)offsets[dg] + excl - lstart;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int loc = wloc + i * 32;
            if (loc < cnt_tile) {
                const uint32_t d = digit_of(k[i], shift, dmask);
                const uint32_t pos = S.local_start[d] + S.warp_hist[warp][d] + r[i];
                S.keys[pos] = k[i];
                S.vals[pos] = kVMode == VM_IOTA ? ValT(uint32_t(base) + uint32_t(loc)) : v[i];
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt_tile; i += kSortThreads) {
            const KeyT kk = S.keys[i];
            const long long o = S.gbase[digit_of(kk, shift, dmask)] + i;
            kout[o] = kk;
            vout[o] = S.vals[i];
        }
        __syncthreads();  // staging, histograms and S.tile are reused by the next tile
    }
}

// Where a partition pass takes its (key, value) pairs: arrays, with the
// values loaded, generated as the index, or generated as the index and the
// previous key (the {ISA, PHI} scatter).  Other sources (pairs computed from
// other arrays) provide the same two members.
template <typename KeyT, typename ValT, int kVMode>
struct ArrayPairs {
    const KeyT *kin;
    const ValT *vin;
    __device__ __forceinline__ void load(int64_t idx, bool valid, KeyT &k, ValT &v) const {
        k = valid ? kin[idx] : KeyT(0);
        if constexpr (kVMode == VM_LOAD) v = valid ? vin[idx] : ValT(0);
        if constexpr (kVMode == VM_IOTA) v = ValT(uint32_t(idx));
        if constexpr (kVMode == VM_IDX_PREV)
            v = uint64_t(uint32_t(idx)) |
                (uint64_t(valid && idx > 0 ? uint32_t(kin[idx - 1]) : 0xFFFFFFFFu) << 32);
    }
    // asks the L2 for pairs [b, b + c) ahead of their use
    __device__ __forceinline__ void prefetch(int64_t b, int64_t c) const {
        const uint32_t kb = uint32_t(c * int64_t(sizeof(KeyT))) & ~15u;
        if (kb && ((uintptr_t(kin + b) & 15) == 0)) prefetch_l2_bulk(kin + b, kb);
        if (kVMode == VM_LOAD) {
            const uint32_t vb = uint32_t(c * int64_t(sizeof(ValT))) & ~15u;
            if (vb && ((uintptr_t(vin + b) & 15) == 0)) prefetch_l2_bulk(vin + b, vb);
        }
    }
};

// One non-stable partition pass, for passes where the order of the elements
// inside a digit bucket does not matter: the bucketed scatters (every bucket
// is read as a set) and the first LSD pass of a sort whose ties may come out
// in any order.  An element's place inside its tile's digit run comes from a
// shared-memory atomic, and the tile's run of each digit is reserved in the
// digit's bucket by one global atomic on the bucket's cursor (cursor[d]
// starts at the bucket's offset): tiles fill their buckets in the order they
// get there, so no tile waits on another (no look-back).  The write is
// staged through shared memory like k_onesweep's.  A persistent grid walks
// the tiles with a grid stride; m_dev, when given, holds the element count.
template <typename KeyT, typename ValT, typename Src>
__global__ void __launch_bounds__(kSortThreads, 4) k_partition(
    Src src, KeyT *__restrict__ kout, ValT *__restrict__ vout, int64_t m, const uint32_t *m_dev, int shift,
    uint32_t dmask, uint32_t *__restrict__ cursor, int *status, int64_t ahead) {
    constexpr int kItems = sort_items<KeyT, ValT>();
    constexpr int kTile = sort_tile<KeyT, ValT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<KeyT, ValT> &S = *reinterpret_cast<OnesweepSmem<KeyT, ValT> *>(smem_raw);
    uint32_t *cnt = S.warp_hist[0];
    const int tid = threadIdx.x;
    if (m_dev) m = int64_t(*m_dev);
    const int64_t ntiles = cdiv(m, kTile);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tid == 0 && ahead > 0) {
            const int64_t b2 = (tile + ahead) * kTile;
            if (b2 < m) src.prefetch(b2, min64(int64_t(kTile), m - b2));
        }
        cnt[tid] = 0;
        __syncthreads();
        const int64_t base = tile * kTile;
        KeyT k[kItems];
        uint32_t r[kItems];
        ValT v[kItems];
        // all items' loads are issued before the first shared-memory atomic
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = base + i * kSortThreads + tid;
            src.load(idx, idx < m, k[i], v[i]);
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = base + i * kSortThreads + tid;
            r[i] = idx < m ? atomicAdd(&cnt[digit_of(k[i], shift, dmask)], 1u) : 0u;
        }
        __syncthreads();
        const int dg = tid;
        const uint32_t total = cnt[dg];
        // this tile's run of digit dg inside the digit's bucket
        const uint32_t run = total ? atomicAdd(&cursor[dg], total) : 0u;
        uint32_t tile_total;
        const uint32_t lstart = block_excl_scan<kSortThreads>(total, S.scratch, &tile_total);
        S.local_start[dg] = lstart;
        S.gbase[dg] = (long long)run - lstart;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = base + i * kSortThreads + tid;
            if (idx < m) {
                const uint32_t pos = S.local_start[digit_of(k[i], shift, dmask)] + r[i];
                S.keys[pos] = k[i];
                S.vals[pos] = v[i];
            }
        }
        __syncthreads();
        const int cnt_tile = int(min64(int64_t(kTile), m - base));
        for (int i = tid; i < cnt_tile; i += kSortThreads) {
            const KeyT kk = S.keys[i];
            const long long o = S.gbase[digit_of(kk, shift, dmask)] + i;
            if (o < 0 || o >= m) {  // counts that did not match the keys (keys meant to be a permutation)
                atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
                continue;
            }
            kout[o] = kk;
            vout[o] = S.vals[i];
        }
        __syncthreads();  // counts and staging are reused by the next tile
    }
}

// The same pass for pairs held in arrays, software-pipelined: while a block
// partitions one tile, the next tile of its grid stride is already on its way
// into shared memory by a bulk (TMA) copy completing on an mbarrier, so the
// DRAM latency of the loads is hidden behind the work of the tile before.
// Whole tiles with 16-byte aligned rows are copied in bulk; a partial or
// unaligned tile is read with plain loads.  Every wait is bounded by the wait
// limit (then LOR_ERR_TIMEOUT, after a bounded wait for the block's own copy
// in flight).
// The staging area of a tile's write is the tile's own input buffer (its
// items are in registers by then; values that are generated, not loaded,
// get one staging array of their own), so that three blocks fit an SM.  For
// 64-bit keys a separate staging area at two blocks per SM measured faster
// (0.93 against 1.06 ms for the 179M-key pass).
template <typename KeyT, typename ValT, int kVMode>
struct PipeSmem {
    static constexpr int kTile = sort_tile<KeyT, ValT>();
    static constexpr bool kLoadV = kVMode == VM_LOAD;
    static constexpr bool kOwnStage = sizeof(KeyT) == 8;
    KeyT in_k[kOwnStage ? 3 : 2][kTile];
    ValT in_v[kLoadV ? (kOwnStage ? 3 : 2) : 1][kTile];
    uint32_t cnt[kRadix];
    uint32_t local_start[kRadix];
    long long gbase[kRadix];
    uint32_t scratch[kSortWarps + 1];
    uint64_t bar[2];
};

template <typename KeyT, typename ValT, int kVMode>
__global__ void __launch_bounds__(kSortThreads, sizeof(KeyT) == 8 ? 2 : 3) k_partition_pipe(
    const KeyT *__restrict__ kin, const ValT *__restrict__ vin, KeyT *__restrict__ kout, ValT *__restrict__ vout,
    int64_t m, const uint32_t *m_dev, int shift, uint32_t dmask, uint32_t *__restrict__ cursor, int *status) {
    using Smem = PipeSmem<KeyT, ValT, kVMode>;
    constexpr int kItems = sort_items<KeyT, ValT>();
    constexpr int kTile = Smem::kTile;
    constexpr bool kLoadV = kVMode == VM_LOAD;
    constexpr uint32_t kBytes = uint32_t(kTile * sizeof(KeyT)) + (kLoadV ? uint32_t(kTile * sizeof(ValT)) : 0u);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    if (m_dev) m = int64_t(*m_dev);
    const int64_t ntiles = cdiv(m, kTile);
    auto bulk_ok = [&](int64_t t) {
        if (t >= ntiles || (t + 1) * kTile > m) return false;
        if (uintptr_t(kin + t * kTile) & 15) return false;
        return !kLoadV || (uintptr_t(vin + t * kTile) & 15) == 0;
    };
    auto issue = [&](int64_t t, int b) {  // one thread
        mbar_arrive_expect_tx(&S.bar[b], kBytes);
        bulk_g2s(S.in_k[b], kin + t * kTile, uint32_t(kTile * sizeof(KeyT)), &S.bar[b]);
        if (kLoadV) bulk_g2s(S.in_v[b], vin + t * kTile, uint32_t(kTile * sizeof(ValT)), &S.bar[b]);
    };
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t limit = wait_limit_ns();
    int64_t tile = blockIdx.x;
    if (tid == 0 && bulk_ok(tile)) issue(tile, 0);
    uint32_t phase = 0;  // bit b: parity of buffer b's next completion
    for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const int64_t nxt = tile + gridDim.x;
        // the other buffer was last read in the previous round, before its
        // closing barrier
        const bool nxt_bulk = bulk_ok(nxt);
        if (tid == 0 && nxt_bulk) {
            fence_proxy_async_smem();
            issue(nxt, b ^ 1);
        }
        S.cnt[tid] = 0;
        const bool bulk = bulk_ok(tile);
        bool failed = false;
        if (bulk) {
            failed = !mbar_wait_bounded(&S.bar[b], (phase >> b) & 1u, limit);
            phase ^= 1u << b;
        }
        if (__syncthreads_or(failed)) {
            // give the block's copies in flight a bounded time to land, then leave
            if (tid == 0) {
                atomicCAS(status, 0, LOR_ERR_TIMEOUT);
                mbar_wait_bounded(&S.bar[b], ((phase >> b) & 1u) ^ 1u, limit);
                if (nxt_bulk) mbar_wait_bounded(&S.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, limit);
            }
            __syncthreads();
            return;
        }
        const int64_t base = tile * kTile;
        KeyT k[kItems];
        uint32_t r[kItems];
        ValT v[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int loc = i * kSortThreads + tid;
            const int64_t idx = base + loc;
            const bool valid = idx < m;
            if (bulk) {
                k[i] = S.in_k[b][loc];
                if constexpr (kVMode == VM_LOAD) v[i] = S.in_v[b][loc];
            } else {
                k[i] = valid ? kin[idx] : KeyT(0);
                if constexpr (kVMode == VM_LOAD) v[i] = valid ? vin[idx] : ValT(0);
            }
            if constexpr (kVMode == VM_IOTA) v[i] = ValT(uint32_t(idx));
            if constexpr (kVMode == VM_IDX_PREV) {
                uint32_t prev = 0xFFFFFFFFu;
                if (valid && idx > 0) prev = (bulk && loc > 0) ? uint32_t(S.in_k[b][loc - 1]) : uint32_t(kin[idx - 1]);
                v[i] = uint64_t(uint32_t(idx)) | (uint64_t(prev) << 32);
            }
            r[i] = valid ? atomicAdd(&S.cnt[digit_of(k[i], shift, dmask)], 1u) : 0u;
        }
        __syncthreads();
        const int dg = tid;
        const uint32_t total = S.cnt[dg];
        // this tile's run of digit dg inside the digit's bucket
        const uint32_t run = total ? atomicAdd(&cursor[dg], total) : 0u;
        uint32_t tile_total;
        const uint32_t lstart = block_excl_scan<kSortThreads>(total, S.scratch, &tile_total);
        S.local_start[dg] = lstart;
        S.gbase[dg] = (long long)run - lstart;
        __syncthreads();  // every item is in registers: the input buffer becomes the staging area
        KeyT *stage_k = S.in_k[Smem::kOwnStage ? 2 : b];
        ValT *stage_v = S.in_v[kLoadV ? (Smem::kOwnStage ? 2 : b) : 0];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = base + i * kSortThreads + tid;
            if (idx < m) {
                const uint32_t pos = S.local_start[digit_of(k[i], shift, dmask)] + r[i];
                stage_k[pos] = k[i];
                stage_v[pos] = v[i];
            }
        }
        __syncthreads();
        const int cnt_tile = int(min64(int64_t(kTile), m - base));
        for (int i = tid; i < cnt_tile; i += kSortThreads) {
            const KeyT kk = stage_k[i];
            const long long o = S.gbase[digit_of(kk, shift, dmask)] + i;
            if (o < 0 || o >= m) {  // counts that did not match the keys (keys meant to be a permutation)
                atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
                continue;
            }
            kout[o] = kk;
            vout[o] = stage_v[i];
        }
        __syncthreads();  // counts and the buffer are reused
    }
}

// Blocks of a pipelined partition pass: as many as fit an SM, times the SMs.
template <typename KeyT, typename ValT, int kVMode>
int partition_pipe_grid(int64_t ntiles, size_t smem) {
    static thread_local int dev = -1, cap = 0;
    int cur = 0;
    LOR_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev) {
        int sms = 0, per = 0;
        LOR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur));
        LOR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_partition_pipe<KeyT, ValT, kVMode>,
                                                                  kSortThreads, smem));
        cap = (per > 0 ? per : 1) * sms;
        dev = cur;
    }
    return int(min64(ntiles > 0 ? ntiles : 1, cap));
}

template <typename KeyT, typename ValT, int kVMode>
int launch_partition_pipe(const KeyT *kin, const ValT *vin, KeyT *kout, ValT *vout, int64_t m, const uint32_t *m_dev,
                          int shift, uint32_t dmask, uint32_t *cursor, int *status, cudaStream_t s) {
    const size_t smem = sizeof(PipeSmem<KeyT, ValT, kVMode>) + 128;
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_partition_pipe<KeyT, ValT, kVMode>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    const int grid = partition_pipe_grid<KeyT, ValT, kVMode>(cdiv(m, sort_tile<KeyT, ValT>()), smem);
    if (grid < 0) return grid;
    k_partition_pipe<KeyT, ValT, kVMode><<<unsigned(grid), kSortThreads, smem, s>>>(kin, vin, kout, vout, m, m_dev,
                                                                                   shift, dmask, cursor, status);
    return LOR_OK;
}

inline int sort_grid_cap();

// Launches k_partition on m pairs from `src` by digit bits [shift, shift +
// width of dmask), consuming `cursor` (the buckets' offsets) as the buckets'
// fill positions.  The caller accounts the launch.
template <typename KeyT, typename ValT, typename Src>
int launch_partition(const Src &src, KeyT *kout, ValT *vout, int64_t m, const uint32_t *m_dev, int shift,
                     uint32_t dmask, uint32_t *cursor, int *status, cudaStream_t s) {
    const size_t smem = sizeof(OnesweepSmem<KeyT, ValT>);
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_partition<KeyT, ValT, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
    const unsigned grid = unsigned(min64(cdiv(m > 0 ? m : 1, sort_tile<KeyT, ValT>()), sort_grid_cap()));
    k_partition<KeyT, ValT, Src><<<grid, kSortThreads, smem, s>>>(src, kout, vout, m, m_dev, shift, dmask, cursor,
                                                                  status, int64_t(grid));
    return LOR_OK;
}

static __global__ void k_iota_u32(uint32_t *__restrict__ v, int64_t m) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) v[i] = uint32_t(i);
}

// Scratch that one sort needs besides the two key/value buffer pairs.
//
// Graph mode (`graph` set) is for work enqueued under CUDA stream capture:
// no call reads anything back to the host, so sorts run every pass (no
// skipping of passes whose digit is the same for all keys), and launches
// whose number of tile claims depends on a count held on the device take a
// counter of their own from `ctr_pool` (zeroed, like the look-back area, at
// the start of the captured work) instead of the running counter.
struct RadixScratch {
    uint32_t *hist = nullptr;          // kMaxPasses * kRadix
    uint32_t *offsets = nullptr;       // kMaxPasses * kRadix
    uint64_t *lookback = nullptr;      // max_tiles * kRadix, zeroed before first use
    unsigned long long *tile_ctr = nullptr;  // zeroed before first use
    unsigned long long tile_base = 0;  // host mirror of *tile_ctr
    uint32_t epoch = 0;                // host counter; 0 is never a valid epoch
    int64_t max_tiles = 0;
    int *status = nullptr;
    cudaStream_t stream = 0;
    bool graph = false;
    unsigned long long *ctr_pool = nullptr;
    int ctr_pool_size = 0, ctr_next = 0;
};

// Resident blocks of a persistent sort pass: four per SM.
inline int sort_grid_cap() {
    static thread_local int dev = -1, cap = 0;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return 4 * 148;
    if (cur != dev) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur) != cudaSuccess || sms <= 0) sms = 148;
        cap = 4 * sms;
        dev = cur;
    }
    return cap;
}

// The tile counter of one launch: the running counter and its host mirror,
// or for a device-sized launch (whose number of claims the host does not
// know) a fresh counter: one from the pool in graph mode, else the running
// counter zeroed before the launch (and again by end_counter after it).
inline int take_counter(RadixScratch &rs, bool device_sized, unsigned long long **ctr,
                        unsigned long long *base) {
    if (rs.graph && device_sized) {
        if (!rs.ctr_pool || rs.ctr_next >= rs.ctr_pool_size) return LOR_ERR_WORKSPACE;
        *ctr = rs.ctr_pool + rs.ctr_next++;
        *base = 0;
    } else if (device_sized) {
        LOR_CUDA_TRY(cudaMemsetAsync(rs.tile_ctr, 0, sizeof(unsigned long long), rs.stream));
        rs.tile_base = 0;
        *ctr = rs.tile_ctr;
        *base = 0;
    } else {
        *ctr = rs.tile_ctr;
        *base = rs.tile_base;
    }
    return LOR_OK;
}

// After a launch that took its counter from take_counter: advances the host
// mirror by the launch's claims, or re-zeroes a running counter that a
// device-sized launch advanced by an unknown amount.
inline int end_counter(RadixScratch &rs, bool device_sized, const unsigned long long *ctr,
                       unsigned long long claims) {
    if (ctr != rs.tile_ctr) return LOR_OK;
    if (device_sized) {
        LOR_CUDA_TRY(cudaMemsetAsync(rs.tile_ctr, 0, sizeof(unsigned long long), rs.stream));
        rs.tile_base = 0;
    } else {
        rs.tile_base += claims;
    }
    return LOR_OK;
}

inline size_t radix_lookback_bytes(int64_t max_m) {
    return size_t(cdiv(max_m > 0 ? max_m : 1, kMinSortTile)) * kRadix * sizeof(uint64_t);
}

// Sort m pairs by bits [begin_bit, end_bit) of the keys.  (k0, v0) hold the
// input; (k1, v1) are same-sized buffers.  On return *kres / *vres point at
// whichever pair holds the sorted result.  When iota_vals is set the values
// are taken to be 0..m-1 and v0 is not read.
// When hist_ready is set the caller has already counted every pass's digits
// into rs.hist (zeroed first), e.g. in the kernel that made the keys.
// When m_dev is given the number of pairs is read from device memory and m
// is only its upper bound (buffer and grid sizes).
// The passes of one sort at kItems keys per thread (see radix_sort_pairs).
template <typename KeyT, int kItems>
int radix_passes(RadixScratch &rs, KeyT *k0, uint32_t *v0, KeyT *k1, uint32_t *v1, int64_t m, int begin_bit,
                 int end_bit, int dbits, int npasses, const uint32_t *hh, bool vals_ready,
                 const uint32_t *m_dev, KeyT **kres, uint32_t **vres, bool ties_any_order) {
    cudaStream_t s = rs.stream;
    constexpr int kTile = kSortThreads * kItems;
    if (cdiv(m, kTile) > rs.max_tiles) return LOR_ERR_WORKSPACE;
    const size_t smem = sizeof(OnesweepSmem<KeyT, uint32_t, kItems>);
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<KeyT, uint32_t, VM_IOTA, kItems>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<KeyT, uint32_t, VM_LOAD, kItems>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    KeyT *ki = k0, *ko = k1;
    uint32_t *vi = v0, *vo = v1;
    const int64_t ntiles = cdiv(m, kTile);
    const unsigned grid = unsigned(min64(ntiles, sort_grid_cap()));
    bool first = true;
    for (int p = 0; p < npasses; ++p) {
        if (hh) {
            bool trivial = false;
            for (int dgt = 0; dgt < kRadix; ++dgt)
                if (int64_t(hh[p * kRadix + dgt]) == m) trivial = true;
            if (trivial) continue;  // every key has the same digit: order unchanged
        }
        const int shift = begin_bit + p * dbits;
        const uint32_t dmask = digit_mask(shift, end_bit, dbits);
        if (first && ties_any_order) {
            // The first pass keeps no earlier order, so when equal keys may come
            // out in any order it need not be stable: a partition pass (no
            // stable ranking, no look-back) on this pass's digit.  The pass's
            // offsets serve as its bucket cursors.
            first = false;
            {
                ProfScope ps(PK_RADIX_PASS, double(m) * (sizeof(KeyT) + (vals_ready ? 4.0 : 0.0) + sizeof(KeyT) + 4),
                             s);
                const int rc = vals_ready
                    ? launch_partition_pipe<KeyT, uint32_t, VM_LOAD>(ki, vi, ko, vo, m, m_dev, shift, dmask,
                                                                      rs.offsets + p * kRadix, rs.status, s)
                    : launch_partition_pipe<KeyT, uint32_t, VM_IOTA>(ki, vi, ko, vo, m, m_dev, shift, dmask,
                                                                      rs.offsets + p * kRadix, rs.status, s);
                if (rc) return rc;
            }
            LOR_LAUNCH_CHECK();
            vals_ready = true;
            KeyT *tk = ki; ki = ko; ko = tk;
            uint32_t *tv = vi; vi = vo; vo = tv;
            continue;
        }
        first = false;
        rs.epoch++;
        unsigned long long *ctr, base;
        int rc = take_counter(rs, m_dev != nullptr, &ctr, &base);
        if (rc) return rc;
        {
            ProfScope ps(PK_RADIX_PASS, double(m) * 2.0 * (sizeof(KeyT) + 4), s);
            if (vals_ready) {
                k_onesweep<KeyT, uint32_t, VM_LOAD, kItems><<<grid, kSortThreads, smem, s>>>(
                    ki, vi, ko, vo, m, m_dev, shift, dmask, rs.offsets + p * kRadix, rs.lookback, ctr, base,
                    rs.epoch, rs.status, prefetch_ahead(ki, vi, grid));
            } else {
                k_onesweep<KeyT, uint32_t, VM_IOTA, kItems><<<grid, kSortThreads, smem, s>>>(
                    ki, vi, ko, vo, m, m_dev, shift, dmask, rs.offsets + p * kRadix, rs.lookback, ctr, base,
                    rs.epoch, rs.status, prefetch_ahead(ki, ki, grid));
            }
        }
        LOR_LAUNCH_CHECK();
        rc = end_counter(rs, m_dev != nullptr, ctr, (unsigned long long)(ntiles + grid));
        if (rc) return rc;
        vals_ready = true;
        KeyT *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    if (!vals_ready) {
        k_iota_u32<<<unsigned(cdiv(m, 256)), 256, 0, s>>>(vi, m);
        LOR_LAUNCH_CHECK();
    }
    *kres = ki;
    *vres = vi;
    return LOR_OK;
}

// Sort m pairs by bits [begin_bit, end_bit) of the keys.  (k0, v0) hold the
// input; (k1, v1) are same-sized buffers.  On return *kres / *vres point at
// whichever pair holds the sorted result.  When iota_vals is set the values
// are taken to be 0..m-1 and v0 is not read.
// When hist_ready is set the caller has already counted every pass's digits
// into rs.hist (zeroed first; digits of tune_config().digit_bits), e.g. in the
// kernel that made the keys.
// When m_dev is given the number of pairs is read from device memory and m
// is only its upper bound (buffer and grid sizes).
// Digit width and keys per thread come from tune_config().
template <typename KeyT>
int radix_sort_pairs(RadixScratch &rs, KeyT *k0, uint32_t *v0, KeyT *k1, uint32_t *v1, int64_t m,
                     int begin_bit, int end_bit, bool iota_vals, KeyT **kres, uint32_t **vres,
                     bool hist_ready = false, const uint32_t *m_dev = nullptr, bool ties_any_order = false) {
    cudaStream_t s = rs.stream;
    *kres = k0;
    *vres = v0;
    if (m <= 0) return LOR_OK;
    const TuneConfig cfg = tune_config();
    const int dbits = cfg.digit_bits;
    const int npasses = int(cdiv(end_bit - begin_bit, dbits));
    if (begin_bit < 0 || end_bit < begin_bit || end_bit > int(8 * sizeof(KeyT)) ||
        npasses > kMaxPasses)
        return LOR_ERR_INVALID_ARG;
    const bool sync_free = rs.graph || m_dev;
    uint32_t hh[kMaxPasses * kRadix];
    if (npasses > 0) {
        if (!hist_ready) {
            LOR_CUDA_TRY(cudaMemsetAsync(rs.hist, 0, sizeof(uint32_t) * npasses * kRadix, s));
            {
                ProfScope ps(PK_RADIX_HIST, double(m) * sizeof(KeyT), s);
                const int grid = int(min64(cdiv(m, 256 * 4), 152 * 8));
                k_radix_hist<KeyT><<<grid, 256, 0, s>>>(k0, m, m_dev, begin_bit, end_bit, npasses, dbits,
                                                        rs.hist);
            }
            LOR_LAUNCH_CHECK();
        }
        k_radix_offsets<<<npasses, kRadix, 0, s>>>(rs.hist, rs.offsets);
        LOR_LAUNCH_CHECK();
        if (!sync_free) {
            LOR_CUDA_TRY(cudaMemcpyAsync(hh, rs.hist, sizeof(uint32_t) * npasses * kRadix,
                                         cudaMemcpyDeviceToHost, s));
            LOR_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    const uint32_t *h = sync_free ? nullptr : hh;
    const int items = sizeof(KeyT) == 8 ? cfg.sort_items_64 : cfg.sort_items_32;
    if (sizeof(KeyT) == 8) {
        if (items == 8)
            return radix_passes<KeyT, 8>(rs, k0, v0, k1, v1, m, begin_bit, end_bit, dbits, npasses, h, !iota_vals,
                                         m_dev, kres, vres, ties_any_order);
        if (items == 16)
            return radix_passes<KeyT, 16>(rs, k0, v0, k1, v1, m, begin_bit, end_bit, dbits, npasses, h, !iota_vals,
                                          m_dev, kres, vres, ties_any_order);
        return radix_passes<KeyT, 12>(rs, k0, v0, k1, v1, m, begin_bit, end_bit, dbits, npasses, h, !iota_vals,
                                      m_dev, kres, vres, ties_any_order);
    }
    if (items == 12)
        return radix_passes<KeyT, 12>(rs, k0, v0, k1, v1, m, begin_bit, end_bit, dbits, npasses, h, !iota_vals,
                                      m_dev, kres, vres, ties_any_order);
    return radix_passes<KeyT, 16>(rs, k0, v0, k1, v1, m, begin_bit, end_bit, dbits, npasses, h, !iota_vals,
                                  m_dev, kres, vres, ties_any_order);
}

// ---- bucketed scatter: dst[key[i]] = val[i] + add for distinct keys in
// [0, bound).  A random 4-byte store costs a DRAM sector; here one radix pass
// on the top 8 bits of the keys groups the pairs by destination window
// (bound / 256 entries), and a streaming pass then writes them: consecutive
// blocks write into the same small window, so the stores combine in L2.
// When m == bound the keys are a permutation of [0, m) (every inverse-array
// scatter of the path): each window then holds exactly bound / 256 keys and
// the pass needs no histogram of them.

// Four pairs per thread (16-byte loads when the four are whole and aligned).
// kDst only names the destination in profiles (0 ranks and other arrays, 1
// the inverse suffix array).
template <int kDst>
__global__ void k_scatter_pairs(const uint32_t *__restrict__ key, const uint32_t *__restrict__ val,
                                       int64_t m, int32_t *__restrict__ dst, int32_t add, int64_t bound,
                                       int *status) {
    const int64_t i0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
    if (i0 >= m) return;
    uint32_t kk[4], vv[4];
    if (i0 + 4 <= m && ((uintptr_t(key + i0) | uintptr_t(val + i0)) & 15) == 0) {
        const uint4 a = *reinterpret_cast<const uint4 *>(key + i0);
        const uint4 b = *reinterpret_cast<const uint4 *>(val + i0);
        kk[0] = a.x; kk[1] = a.y; kk[2] = a.z; kk[3] = a.w;
        vv[0] = b.x; vv[1] = b.y; vv[2] = b.z; vv[3] = b.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            kk[u] = i0 + u < m ? key[i0 + u] : 0xFFFFFFFFu;
            vv[u] = i0 + u < m ? val[i0 + u] : 0u;
        }
    }
    bool bad = false;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (i0 + u >= m) break;
        if (int64_t(kk[u]) >= bound) {
            bad = true;
            continue;
        }
        dst[kk[u]] = int32_t(vv[u]) + add;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
}

// keys/vals: inputs (vals == nullptr means 0..m-1).  kbuf, vbuf0, vbuf1:
// caller scratch of m entries each (vbuf0 receives the input values when they
// are generated).  The caller accounts the scatter kernel's launch.
// One partition pass of m keys by bits [lo, top) (top - lo <= 8): histogram,
// offsets and k_partition.  No host synchronisation.
// Keys that are a permutation of [0, m) fill every bucket of 2^lo keys
// exactly: its start is known without counting.
static __global__ void k_perm_offsets(uint32_t *__restrict__ offsets, int lo, int64_t m) {
    const int64_t o = int64_t(threadIdx.x) << lo;
    offsets[threadIdx.x] = uint32_t(o < m ? o : m);
}

// (perm: the keys are a permutation of [0, m), as for every inverse-array
// scatter here; then the bucket starts need no histogram.)
template <typename ValT, int kVMode>
int partition_pass(RadixScratch &rs, const uint32_t *keys, const ValT *vals, int64_t m, int lo, int top,
                   uint32_t *kout, ValT *vout, bool perm = false) {
    cudaStream_t s = rs.stream;
    if (perm) {
        k_perm_offsets<<<1, kRadix, 0, s>>>(rs.offsets, lo, m);
        LOR_LAUNCH_CHECK();
    } else {
        LOR_CUDA_TRY(cudaMemsetAsync(rs.hist, 0, sizeof(uint32_t) * kRadix, s));
        {
            ProfScope ps(PK_RADIX_HIST, double(m) * 4, s);
            const int grid = int(min64(cdiv(m, 256 * 4), 152 * 8));
            k_radix_hist<uint32_t><<<grid, 256, 0, s>>>(keys, m, nullptr, lo, top, 1, kRadixBits, rs.hist);
        }
        LOR_LAUNCH_CHECK();
        k_radix_offsets<<<1, kRadix, 0, s>>>(rs.hist, rs.offsets);
        LOR_LAUNCH_CHECK();
    }
    {
        ProfScope ps(PK_RADIX_PASS, double(m) * (4 + (kVMode == VM_LOAD ? sizeof(ValT) : 0) + 4 + sizeof(ValT)),
                     s);
        // the offsets are consumed as the buckets' cursors
        const int rc = launch_partition_pipe<uint32_t, ValT, kVMode>(keys, vals, kout, vout, m, nullptr, lo,
                                                                     digit_mask(lo, top), rs.offsets, rs.status, s);
        if (rc) return rc;
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

inline int bucketed_scatter(RadixScratch &rs, const uint32_t *keys, const uint32_t *vals, int64_t m,
                            int64_t bound, uint32_t *kbuf, uint32_t *vbuf0, uint32_t *vbuf1,
                            int32_t *dst, int32_t add, int kind = PK_RANK_SCATTER) {
    (void)vbuf1;
    if (m <= 0) return LOR_OK;
    const int top = bit_width_u64(uint64_t(bound > 1 ? bound - 1 : 1));
    const int lo = top > kRadixBits ? top - kRadixBits : 0;
    const int rc = vals ? partition_pass<uint32_t, VM_LOAD>(rs, keys, vals, m, lo, top, kbuf, vbuf0, m == bound)
                        : partition_pass<uint32_t, VM_IOTA>(rs, keys, nullptr, m, lo, top, kbuf, vbuf0, m == bound);
    if (rc) return rc;
    {
        ProfScope ps(kind, double(m) * 12, rs.stream);
        auto kern = kind == PK_ISA_SCATTER ? k_scatter_pairs<1> : k_scatter_pairs<0>;
        kern<<<unsigned(cdiv(cdiv(m, 4), 256)), 256, 0, rs.stream>>>(kbuf, vbuf0, m, dst, add, bound,
                                                                      rs.status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

// ---- the same bucketing for {ISA, PHI}: ip[SA[k]] = {k, SA[k-1]}.  One
// partition pass on the top 8 bits of SA[k] whose 64-bit values are generated
// in the pass (k and the previous key), then a streaming 8-byte scatter.

static __global__ void k_scatter_isa_phi(const uint32_t *__restrict__ key, const uint64_t *__restrict__ val,
                                         int64_t m, int2 *__restrict__ ip, int64_t bound, int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t r = key[i];
    if (int64_t(r) >= bound) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    const uint64_t v = val[i];
    ip[r] = make_int2(int32_t(uint32_t(v)), int32_t(uint32_t(v >> 32)));
}

// sa: m entries (a permutation of [0, bound)); kbuf: m uint32 scratch; vbuf:
// m uint64 scratch.
inline int bucketed_isa_phi(RadixScratch &rs, const int32_t *sa, int64_t m, int64_t bound, uint32_t *kbuf,
                            uint64_t *vbuf, int2 *ip) {
    if (m <= 0) return LOR_OK;
    const int top = bit_width_u64(uint64_t(bound > 1 ? bound - 1 : 1));
    const int lo = top > kRadixBits ? top - kRadixBits : 0;
    const int rc = partition_pass<uint64_t, VM_IDX_PREV>(rs, reinterpret_cast<const uint32_t *>(sa), nullptr, m,
                                                          lo, top, kbuf, vbuf, m == bound);
    if (rc) return rc;
    {
        ProfScope ps(PK_ISA_SCATTER, double(m) * 20, rs.stream);
        k_scatter_isa_phi<<<unsigned(cdiv(m, 256)), 256, 0, rs.stream>>>(kbuf, vbuf, m, ip, bound, rs.status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

}  // namespace lor
