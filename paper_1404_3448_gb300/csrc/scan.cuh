// scan.cuh -- order-preserving tile compaction and naming by single-pass
// decoupled look-back scans (bounded waits), shared by the DC3 levels and the
// batched pipeline.
#pragma once

#include "common.cuh"

namespace lor {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Loads the N consecutive items p[base .. base+N) of one thread (entries at
// or past m read as `fill`): 16-byte loads when the run is whole and aligned.
template <typename T, int N>
__device__ __forceinline__ void load_run(const T *__restrict__ p, int64_t base, int64_t m, T fill, T (&out)[N]) {
    static_assert((N * sizeof(T)) % 16 == 0, "run must be whole 16-byte chunks");
    if (base + N <= m && ((uintptr_t)(p + base) & 15) == 0) {
        const int4 *q = reinterpret_cast<const int4 *>(p + base);
        int4 *o = reinterpret_cast<int4 *>(out);
#pragma unroll
        for (int c = 0; c < int(N * sizeof(T) / 16); ++c) o[c] = q[c];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = base + i < m ? p[base + i] : fill;
    }
}

// Stores the N consecutive items of one thread at p[base ..], those below m.
template <typename T, int N>
__device__ __forceinline__ void store_run(T *__restrict__ p, int64_t base, int64_t m, const T (&v)[N]) {
    static_assert((N * sizeof(T)) % 16 == 0, "run must be whole 16-byte chunks");
    if (base + N <= m && ((uintptr_t)(p + base) & 15) == 0) {
        int4 *q = reinterpret_cast<int4 *>(p + base);
        const int4 *o = reinterpret_cast<const int4 *>(v);
#pragma unroll
        for (int c = 0; c < int(N * sizeof(T) / 16); ++c) q[c] = o[c];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (base + i < m) p[base + i] = v[i];
    }
}

// ---- generic order-preserving tile compaction and naming (look-back scans)

// Every kernel below handles kScanTile consecutive items per block (blocked:
// kScanItems per thread), claims its tile from the running counter, scans its
// predicate and walks back over predecessor tiles for the global offset.
template <typename Pred, typename Emit>
__device__ __forceinline__ void tile_compact(int64_t m, Pred pred, Emit emit, uint64_t *lb,
                                             unsigned long long *ctr, unsigned long long tile_base,
                                             uint32_t epoch, int *status, uint32_t *count,
                                             int64_t ntiles) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < m && pred(j)) {
            flags |= 1u << i;
            cnt++;
        }
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
        if ((flags >> i) & 1u) emit(base + i, o++);
}

// name(j) = number of j' <= j where NewName(j') holds (NewName(0) must hold).
template <typename NewName, typename Emit>
__device__ __forceinline__ void tile_names(int64_t m, NewName is_new, Emit emit, uint32_t *n_names,
                                           uint64_t *lb, unsigned long long *ctr,
                                           unsigned long long tile_base, uint32_t epoch, int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < m && is_new(j)) {
            flags |= 1u << i;
            cnt++;
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
            emit(j, name);
            if (j == m - 1) *n_names = name;
        }
    }
}

// ---- the same scans over a count held on the device
//
// For work enqueued without host round trips (CUDA graph capture): the item
// count is read from m_dev, a small grid of resident blocks claims tiles from
// `ctr` (a counter of this launch alone, zeroed beforehand) until it draws
// one past the last tile, and an empty input still writes its count (0).

template <typename Pred, typename Emit>
__device__ __forceinline__ void tile_compact_dyn(const uint32_t *m_dev, Pred pred, Emit emit, uint64_t *lb,
                                                 unsigned long long *ctr, uint32_t epoch, int *status,
                                                 uint32_t *count) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    const int64_t m = int64_t(*m_dev);
    const int64_t ntiles = cdiv(m, kScanTile);
    if (ntiles == 0) {
        if (count && blockIdx.x == 0 && tid == 0) *count = 0;
        return;
    }
    for (;;) {
        if (tid == 0) s_tile = (long long)atomicAdd(ctr, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;  // uniform over the block
        const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
        uint32_t flags = 0, cnt = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t j = base + i;
            if (j < m && pred(j)) {
                flags |= 1u << i;
                cnt++;
            }
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
            if ((flags >> i) & 1u) emit(base + i, o++);
        __syncthreads();  // s_tile and s_prefix are reused by the next tile
    }
}

template <typename NewName, typename Emit>
__device__ __forceinline__ void tile_names_dyn(const uint32_t *m_dev, NewName is_new, Emit emit, uint64_t *lb,
                                               unsigned long long *ctr, uint32_t epoch, int *status) {
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    const int64_t m = int64_t(*m_dev);
    const int64_t ntiles = cdiv(m, kScanTile);
    for (;;) {
        if (tid == 0) s_tile = (long long)atomicAdd(ctr, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;  // uniform over the block
        const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
        uint32_t flags = 0, cnt = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t j = base + i;
            if (j < m && is_new(j)) {
                flags |= 1u << i;
                cnt++;
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
                emit(j, name);
            }
        }
        __syncthreads();
    }
}

// Resident blocks of a scan over a device-held count: eight per SM.
inline unsigned scan_grid_cap() {
    static thread_local int dev = -1;
    static thread_local unsigned cap = 0;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return 8 * 148;
    if (cur != dev) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur) != cudaSuccess || sms <= 0) sms = 148;
        cap = unsigned(8 * sms);
        dev = cur;
    }
    return cap;
}

}  // namespace lor
