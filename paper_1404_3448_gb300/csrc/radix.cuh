// radix.cuh -- stable LSD radix sort of (key, uint32 value) pairs.
//
// The paper's DC3 sorts its sample triples and nonsample pairs with an LSD
// radix sort (Section 4, Algorithm 1: one 1-bit split per pass, block-local
// chunks merged afterwards).  Here one pass moves 8 bits: an up-front
// histogram kernel counts every pass's digits in one read of the keys, and
// each pass is a single "onesweep" kernel -- a block ranks its tile of keys
// with warp match/popc, learns the global offset of each digit from its
// predecessors by decoupled look-back (bounded waits), and scatters through
// shared memory so that every digit run is written contiguously.
#pragma once

#include "common.cuh"

namespace lor {

constexpr int kRadixBits = 8;
constexpr int kRadix = 256;
constexpr int kSortThreads = 256;  // == kRadix: one thread per digit in the look-back
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxPasses = 8;  // 64-bit keys

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
constexpr int kMinSortTile = kSortThreads * 12;

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift, uint32_t mask = 0xFFu) {
    return uint32_t(k >> shift) & mask;
}
// Digit mask of the pass starting at `shift` when the key ends at end_bit.
__host__ __device__ __forceinline__ uint32_t digit_mask(int shift, int end_bit) {
    const int w = end_bit - shift < kRadixBits ? end_bit - shift : kRadixBits;
    return (1u << w) - 1u;
}

// Digit histograms of every pass in one read of the keys.  Counts go to
// shared-memory atomics; when all 32 lanes of a warp hold the same digit (low
// entropy passes) one lane adds 32 instead.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_radix_hist(const KeyT *__restrict__ keys, int64_t m,
                                                    int begin_bit, int end_bit, int npasses,
                                                    uint32_t *__restrict__ hist) {
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
            const int sft = begin_bit + p * kRadixBits;
            const uint32_t dm = digit_mask(sft, end_bit);
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

template <typename KeyT, typename ValT>
struct OnesweepSmem {
    KeyT keys[sort_tile<KeyT, ValT>()];
    ValT vals[sort_tile<KeyT, ValT>()];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t local_start[kRadix];
    long long gbase[kRadix];
    uint32_t scratch[kSortWarps + 1];
    long long tile;
};

// One LSD pass over digit (shift .. shift+7).  Tiles are claimed in launch
// order from a running counter, so every predecessor a block waits on is
// already resident; each wait is still bounded by kSpinLimitNs.
template <typename KeyT, typename ValT, int kVMode>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(
    const KeyT *__restrict__ kin, const ValT *__restrict__ vin, KeyT *__restrict__ kout,
    ValT *__restrict__ vout, int64_t m, int shift, uint32_t dmask,
    const uint32_t *__restrict__ offsets,
    uint64_t *__restrict__ lookback, unsigned long long *tile_ctr, unsigned long long tile_base,
    uint32_t epoch, int *status, int64_t ahead) {
    constexpr int kItems = sort_items<KeyT, ValT>();
    constexpr int kTile = sort_tile<KeyT, ValT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<KeyT, ValT> &S = *reinterpret_cast<OnesweepSmem<KeyT, ValT> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        S.tile = (long long)(atomicAdd(tile_ctr, 1ull) - tile_base);
        const int64_t b2 = (S.tile + ahead) * kTile;
        if (ahead > 0 && b2 < m) {
            const int64_t c2 = min64(int64_t(kTile), m - b2);
            const uint32_t kb = uint32_t(c2 * int64_t(sizeof(KeyT))) & ~15u;
            if (kb) prefetch_l2_bulk(kin + b2, kb);
            if (kVMode == VM_LOAD) {
                const uint32_t vb = uint32_t(c2 * int64_t(sizeof(ValT))) & ~15u;
                if (vb) prefetch_l2_bulk(vin + b2, vb);
            }
        }
    }
    for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&S.warp_hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = S.tile;
    const int64_t base = tile * kTile;
    const int64_t wbase = base + int64_t(warp) * (kItems * 32);

    KeyT k[kItems];
    ValT v[kItems];
    uint32_t r[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = wbase + i * 32 + lane;
        const bool valid = idx < m;
        k[i] = valid ? kin[idx] : KeyT(0);
        if constexpr (kVMode == VM_LOAD) v[i] = valid ? vin[idx] : ValT(0);
        if constexpr (kVMode == VM_IDX_PREV)
            v[i] = uint64_t(uint32_t(idx)) |
                   (uint64_t(valid && idx > 0 ? uint32_t(kin[idx - 1]) : 0xFFFFFFFFu) << 32);
    }
    // Stable rank inside the warp: items in order, lanes in order.  Slots
    // past the end of the input use digit 256 and are never counted.
    uint32_t *wh = S.warp_hist[warp];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const bool valid = wbase + i * 32 + lane < m;
        const uint32_t d = valid ? digit_of(k[i], shift, dmask) : 0x100u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lt = __popc(peers & lanemask_lt());
        const uint32_t cnt = valid ? wh[d] : 0u;
        r[i] = cnt + lt;
        __syncwarp();
        if (valid && lt == 0) wh[d] = cnt + __popc(peers);
        __syncwarp();
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

    // Decoupled look-back, one digit per thread.
    uint32_t excl = 0;
    uint64_t *lb = lookback;
    if (tile == 0) {
        st_volatile_u64(&lb[dg], lb_pack(epoch, kFlagIncl, total));
    } else {
        st_volatile_u64(&lb[tile * kRadix + dg], lb_pack(epoch, kFlagAgg, total));
        int64_t j = tile - 1;
        const uint64_t t0 = global_ns();
        while (j >= 0) {
            const uint64_t w = ld_volatile_u64(&lb[j * kRadix + dg]);
            if (lb_epoch(w) != epoch || lb_flag(w) == 0) {
                if (global_ns() - t0 > kSpinLimitNs) {
                    atomicCAS(status, 0, LOR_ERR_TIMEOUT);
                    break;
                }
                continue;
            }
            excl += lb_value(w);
            if (lb_flag(w) == kFlagIncl) break;
            --j;
        }
        st_volatile_u64(&lb[tile * kRadix + dg], lb_pack(epoch, kFlagIncl, excl + total));
    }
    S.gbase[dg] = (long long)offsets[dg] + excl - lstart;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = wbase + i * 32 + lane;
        if (idx < m) {
            const uint32_t d = digit_of(k[i], shift, dmask);
            const uint32_t pos = S.local_start[d] + S.warp_hist[warp][d] + r[i];
            S.keys[pos] = k[i];
            S.vals[pos] = kVMode == VM_IOTA ? ValT(uint32_t(idx)) : v[i];
        }
    }
    __syncthreads();
    const int cnt_tile = int(min64(int64_t(kTile), m - base));
    for (int i = tid; i < cnt_tile; i += kSortThreads) {
        const KeyT kk = S.keys[i];
        const long long o = S.gbase[digit_of(kk, shift, dmask)] + i;
        kout[o] = kk;
        vout[o] = S.vals[i];
    }
}

// One non-stable partition pass (for the bucketed scatters, where the order
// inside a bucket does not matter): an element's place inside its tile's
// digit run comes from a shared-memory atomic instead of the stable warp
// ranking; the look-back and the staged write are those of k_onesweep.
template <typename ValT, int kVMode>
__global__ void __launch_bounds__(kSortThreads, 4) k_partition(
    const uint32_t *__restrict__ kin, const ValT *__restrict__ vin, uint32_t *__restrict__ kout,
    ValT *__restrict__ vout, int64_t m, int shift, uint32_t dmask, const uint32_t *__restrict__ offsets,
    uint64_t *__restrict__ lookback, unsigned long long *tile_ctr, unsigned long long tile_base,
    uint32_t epoch, int *status, int64_t ahead) {
    constexpr int kItems = sort_items<uint32_t, ValT>();
    constexpr int kTile = sort_tile<uint32_t, ValT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<uint32_t, ValT> &S = *reinterpret_cast<OnesweepSmem<uint32_t, ValT> *>(smem_raw);
    uint32_t *cnt = S.warp_hist[0];
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.tile = (long long)(atomicAdd(tile_ctr, 1ull) - tile_base);
        const int64_t b2 = (S.tile + ahead) * kTile;
        if (ahead > 0 && b2 < m) {
            const int64_t c2 = min64(int64_t(kTile), m - b2);
            const uint32_t kb = uint32_t(c2 * 4) & ~15u;
            if (kb) prefetch_l2_bulk(kin + b2, kb);
            if (kVMode == VM_LOAD) {
                const uint32_t vb = uint32_t(c2 * int64_t(sizeof(ValT))) & ~15u;
                if (vb) prefetch_l2_bulk(vin + b2, vb);
            }
        }
    }
    cnt[tid] = 0;
    __syncthreads();
    const int64_t tile = S.tile;
    const int64_t base = tile * kTile;
    uint32_t k[kItems], r[kItems];
    ValT v[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + i * kSortThreads + tid;
        const bool valid = idx < m;
        k[i] = valid ? kin[idx] : 0u;
        if constexpr (kVMode == VM_LOAD) v[i] = valid ? vin[idx] : ValT(0);
        if constexpr (kVMode == VM_IOTA) v[i] = ValT(uint32_t(idx));
        if constexpr (kVMode == VM_IDX_PREV)
            v[i] = uint64_t(uint32_t(idx)) |
                   (uint64_t(valid && idx > 0 ? kin[idx - 1] : 0xFFFFFFFFu) << 32);
        r[i] = valid ? atomicAdd(&cnt[digit_of(k[i], shift, dmask)], 1u) : 0u;
    }
    __syncthreads();
    const int dg = tid;
    const uint32_t total = cnt[dg];
    uint32_t tile_total;
    const uint32_t lstart = block_excl_scan<kSortThreads>(total, S.scratch, &tile_total);
    S.local_start[dg] = lstart;
    uint32_t excl = 0;
    uint64_t *lb = lookback;
    if (tile == 0) {
        st_volatile_u64(&lb[dg], lb_pack(epoch, kFlagIncl, total));
    } else {
        st_volatile_u64(&lb[tile * kRadix + dg], lb_pack(epoch, kFlagAgg, total));
        int64_t j = tile - 1;
        const uint64_t t0 = global_ns();
        while (j >= 0) {
            const uint64_t w = ld_volatile_u64(&lb[j * kRadix + dg]);
            if (lb_epoch(w) != epoch || lb_flag(w) == 0) {
                if (global_ns() - t0 > kSpinLimitNs) {
                    atomicCAS(status, 0, LOR_ERR_TIMEOUT);
                    break;
                }
                continue;
            }
            excl += lb_value(w);
            if (lb_flag(w) == kFlagIncl) break;
            --j;
        }
        st_volatile_u64(&lb[tile * kRadix + dg], lb_pack(epoch, kFlagIncl, excl + total));
    }
    S.gbase[dg] = (long long)offsets[dg] + excl - lstart;
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
        const uint32_t kk = S.keys[i];
        const long long o = S.gbase[digit_of(kk, shift, dmask)] + i;
        kout[o] = kk;
        vout[o] = S.vals[i];
    }
}

static __global__ void k_iota_u32(uint32_t *__restrict__ v, int64_t m) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) v[i] = uint32_t(i);
}

// Scratch that one sort needs besides the two key/value buffer pairs.
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
};

inline size_t radix_lookback_bytes(int64_t max_m) {
    return size_t(cdiv(max_m > 0 ? max_m : 1, kMinSortTile)) * kRadix * sizeof(uint64_t);
}

// Sort m pairs by bits [begin_bit, end_bit) of the keys.  (k0, v0) hold the
// input; (k1, v1) are same-sized buffers.  On return *kres / *vres point at
// whichever pair holds the sorted result.  When iota_vals is set the values
// are taken to be 0..m-1 and v0 is not read.
// When hist_ready is set the caller has already counted every pass's digits
// into rs.hist (zeroed first), e.g. in the kernel that made the keys.
template <typename KeyT>
int radix_sort_pairs(RadixScratch &rs, KeyT *k0, uint32_t *v0, KeyT *k1, uint32_t *v1, int64_t m,
                     int begin_bit, int end_bit, bool iota_vals, KeyT **kres, uint32_t **vres,
                     bool hist_ready = false) {
    cudaStream_t s = rs.stream;
    *kres = k0;
    *vres = v0;
    if (m <= 0) return LOR_OK;
    const int npasses = int(cdiv(end_bit - begin_bit, kRadixBits));
    if (begin_bit < 0 || end_bit < begin_bit || end_bit > int(8 * sizeof(KeyT)) ||
        npasses > kMaxPasses)
        return LOR_ERR_INVALID_ARG;
    if (cdiv(m, sort_tile<KeyT, uint32_t>()) > rs.max_tiles) return LOR_ERR_WORKSPACE;
    uint32_t hh[kMaxPasses * kRadix];
    if (npasses > 0) {
        if (!hist_ready) {
            LOR_CUDA_TRY(cudaMemsetAsync(rs.hist, 0, sizeof(uint32_t) * npasses * kRadix, s));
            {
                ProfScope ps(PK_RADIX_HIST, double(m) * sizeof(KeyT), s);
                const int grid = int(min64(cdiv(m, 256 * 4), 152 * 8));
                k_radix_hist<KeyT><<<grid, 256, 0, s>>>(k0, m, begin_bit, end_bit, npasses, rs.hist);
            }
            LOR_LAUNCH_CHECK();
        }
        k_radix_offsets<<<npasses, kRadix, 0, s>>>(rs.hist, rs.offsets);
        LOR_LAUNCH_CHECK();
        LOR_CUDA_TRY(cudaMemcpyAsync(hh, rs.hist, sizeof(uint32_t) * npasses * kRadix,
                                     cudaMemcpyDeviceToHost, s));
        LOR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const size_t smem = sizeof(OnesweepSmem<KeyT, uint32_t>);
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<KeyT, uint32_t, VM_IOTA>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<KeyT, uint32_t, VM_LOAD>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    KeyT *ki = k0, *ko = k1;
    uint32_t *vi = v0, *vo = v1;
    bool vals_ready = !iota_vals;
    const int64_t ntiles = cdiv(m, sort_tile<KeyT, uint32_t>());
    for (int p = 0; p < npasses; ++p) {
        bool trivial = false;
        for (int dgt = 0; dgt < kRadix; ++dgt)
            if (int64_t(hh[p * kRadix + dgt]) == m) trivial = true;
        if (trivial) continue;  // every key has the same digit: order unchanged
        const int shift = begin_bit + p * kRadixBits;
        rs.epoch++;
        {
            ProfScope ps(PK_RADIX_PASS, double(m) * 2.0 * (sizeof(KeyT) + 4), s);
            if (vals_ready)
                k_onesweep<KeyT, uint32_t, VM_LOAD><<<unsigned(ntiles), kSortThreads, smem, s>>>(
                    ki, vi, ko, vo, m, shift, digit_mask(shift, end_bit), rs.offsets + p * kRadix,
                    rs.lookback, rs.tile_ctr, rs.tile_base, rs.epoch, rs.status, prefetch_ahead(ki, vi));
            else
                k_onesweep<KeyT, uint32_t, VM_IOTA><<<unsigned(ntiles), kSortThreads, smem, s>>>(
                    ki, vi, ko, vo, m, shift, digit_mask(shift, end_bit), rs.offsets + p * kRadix,
                    rs.lookback, rs.tile_ctr, rs.tile_base, rs.epoch, rs.status, prefetch_ahead(ki, ki));
        }
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
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

// ---- bucketed scatter: dst[key[i]] = val[i] + add for distinct keys in
// [0, bound).  A random 4-byte store costs a DRAM sector; here one radix pass
// on the top 8 bits of the keys groups the pairs by destination window
// (bound / 256 entries), and a streaming pass then writes them: consecutive
// blocks write into the same small window, so the stores combine in L2.

static __global__ void k_scatter_pairs(const uint32_t *__restrict__ key, const uint32_t *__restrict__ val,
                                       int64_t m, int32_t *__restrict__ dst, int32_t add, int64_t bound,
                                       int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t r = key[i];
    if (int64_t(r) >= bound) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    dst[r] = int32_t(val[i]) + add;
}

// keys/vals: inputs (vals == nullptr means 0..m-1).  kbuf, vbuf0, vbuf1:
// caller scratch of m entries each (vbuf0 receives the input values when they
// are generated).  The caller accounts the scatter kernel's launch.
// One partition pass of m keys by bits [lo, top) (top - lo <= 8): histogram,
// offsets and k_partition.  No host synchronisation.
template <typename ValT, int kVMode>
int partition_pass(RadixScratch &rs, const uint32_t *keys, const ValT *vals, int64_t m, int lo, int top,
                   uint32_t *kout, ValT *vout) {
    cudaStream_t s = rs.stream;
    if (cdiv(m, sort_tile<uint32_t, ValT>()) > rs.max_tiles) return LOR_ERR_WORKSPACE;
    LOR_CUDA_TRY(cudaMemsetAsync(rs.hist, 0, sizeof(uint32_t) * kRadix, s));
    {
        ProfScope ps(PK_RADIX_HIST, double(m) * 4, s);
        const int grid = int(min64(cdiv(m, 256 * 4), 152 * 8));
        k_radix_hist<uint32_t><<<grid, 256, 0, s>>>(keys, m, lo, top, 1, rs.hist);
    }
    LOR_LAUNCH_CHECK();
    k_radix_offsets<<<1, kRadix, 0, s>>>(rs.hist, rs.offsets);
    LOR_LAUNCH_CHECK();
    const size_t smem = sizeof(OnesweepSmem<uint32_t, ValT>);
    LOR_CUDA_TRY(cudaFuncSetAttribute(k_partition<ValT, kVMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
    const int64_t ntiles = cdiv(m, sort_tile<uint32_t, ValT>());
    rs.epoch++;
    {
        ProfScope ps(PK_RADIX_PASS, double(m) * (4 + (kVMode == VM_LOAD ? sizeof(ValT) : 0) + 4 + sizeof(ValT)),
                     s);
        k_partition<ValT, kVMode><<<unsigned(ntiles), kSortThreads, smem, s>>>(
            keys, vals, kout, vout, m, lo, digit_mask(lo, top), rs.offsets, rs.lookback, rs.tile_ctr,
            rs.tile_base, rs.epoch, rs.status, prefetch_ahead(keys, kVMode == VM_LOAD ? (const void *)vals : keys));
    }
    LOR_LAUNCH_CHECK();
    rs.tile_base += (unsigned long long)ntiles;
    return LOR_OK;
}

inline int bucketed_scatter(RadixScratch &rs, const uint32_t *keys, const uint32_t *vals, int64_t m,
                            int64_t bound, uint32_t *kbuf, uint32_t *vbuf0, uint32_t *vbuf1,
                            int32_t *dst, int32_t add) {
    (void)vbuf1;
    if (m <= 0) return LOR_OK;
    const int top = bit_width_u64(uint64_t(bound > 1 ? bound - 1 : 1));
    const int lo = top > kRadixBits ? top - kRadixBits : 0;
    const int rc = vals ? partition_pass<uint32_t, VM_LOAD>(rs, keys, vals, m, lo, top, kbuf, vbuf0)
                        : partition_pass<uint32_t, VM_IOTA>(rs, keys, nullptr, m, lo, top, kbuf, vbuf0);
    if (rc) return rc;
    {
        ProfScope ps(PK_RANK_SCATTER, double(m) * 12, rs.stream);
        k_scatter_pairs<<<unsigned(cdiv(m, 256)), 256, 0, rs.stream>>>(kbuf, vbuf0, m, dst, add, bound,
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
                                                          lo, top, kbuf, vbuf);
    if (rc) return rc;
    {
        ProfScope ps(PK_ISA_SCATTER, double(m) * 20, rs.stream);
        k_scatter_isa_phi<<<unsigned(cdiv(m, 256)), 256, 0, rs.stream>>>(kbuf, vbuf, m, ip, bound, rs.status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

}  // namespace lor
