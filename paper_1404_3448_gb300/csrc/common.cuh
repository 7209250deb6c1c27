// common.cuh -- shared device/host helpers of liblor (status word, launch
// accounting, kernel timing hooks, bounded waits, block scans).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "lor.h"

namespace lor {

// ---------------------------------------------------------------- sizes

constexpr int kWarp = 32;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline int bit_width_u64(uint64_t v) {  // number of bits needed to hold v
    int b = 0;
    while (v) { b++; v >>= 1; }
    return b;
}

// ---------------------------------------------------------------- host side

// Launch accounting and kernel timing (defined in abi.cu).
void note_launch();
// Stream capture on this thread: launches are counted for the graph, not run.
void capture_begin();
unsigned long long capture_end();  // kernels captured since capture_begin
void note_graph_launches(unsigned long long kernels);
enum ProfKind {
    PK_ENCODE = 0,
    PK_SAMPLE_KEYS,
    PK_RADIX_HIST,
    PK_RADIX_PASS,
    PK_NAMING,
    PK_RANK_SCATTER,
    PK_NONSAMPLE,
    PK_MERGE,
    PK_ISA_SCATTER,
    PK_KASAI,
    PK_OVERLAP_SCAN,
    PK_OVERLAP_COLLECT,
    PK_RMQ_LEVEL,
    PK_RMQ_QUERY,
    PK_OTHER,
    PK_COUNT
};
bool prof_enabled();

// Launch parameters picked by the autotuner (lor_autotune_batch) or set with
// lor_tune_set; every value gives the same results, only the speed differs.
// A call reads the configuration once when it starts (a CUDA graph keeps the
// one it was captured with).
struct TuneConfig {
    int digit_bits = 8;        // radix digit width of the sorts, 5..8 bits
    int level0_key_bits = 48;  // width of the level-0 sample keys (the symbols named at level 0)
    int sort_items_64 = 12;    // keys per thread of a sort pass over 64-bit keys: 8, 12 or 16
    int sort_items_32 = 16;    // ... over 32-bit keys: 12 or 16
    int merge_items = 4;       // merged suffixes per thread of the Step-3 merge: 2, 4 or 8 (512, 256, 128 threads)
};
TuneConfig tune_config();
// Records an event pair around one launch when profiling is on.
struct ProfScope {
    int slot = -1;
    cudaStream_t stream;
    ProfScope(int kind, double bytes, cudaStream_t s);
    ~ProfScope();
};

// Scoped device status helpers: every translation unit owns one status word.
#define LOR_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return LOR_ERR_CUDA;         \
    } while (0)

#define LOR_LAUNCH_CHECK()                                  \
    do {                                                    \
        lor::note_launch();                                 \
        cudaError_t _e = cudaPeekAtLastError();             \
        if (_e != cudaSuccess) return LOR_ERR_CUDA;         \
    } while (0)

// ---------------------------------------------------------------- device side

// Asks the L2 to fetch [p, p + bytes) ahead of its use (p 16-byte aligned,
// bytes a multiple of 16): a hint with no effect on results.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Asks the L2 for the whole 16-byte groups inside [a, e): a hint that touches
// nothing outside the range.
template <typename T>
__device__ __forceinline__ void prefetch_inside(const T *a, const T *e) {
    const uintptr_t lo = (uintptr_t(a) + 15) & ~uintptr_t(15), hi = uintptr_t(e) & ~uintptr_t(15);
    if (hi > lo && hi - lo < (uintptr_t(1) << 31)) prefetch_l2_bulk((const void *)lo, uint32_t(hi - lo));
}

// Tiles a radix pass asks the L2 to fetch ahead of the one it works on: the
// number of tiles resident at once (four 256-thread blocks per SM, or the
// grid of a persistent pass), so that the data of the tile a block takes next
// is already in L2.  0 when a buffer is not 16-byte aligned.
inline int64_t prefetch_ahead(const void *a, const void *b, int64_t resident = 0) {
    if ((uintptr_t(a) | uintptr_t(b)) & 15) return 0;
    if (resident > 0) return resident;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return int64_t(4) * sms;
}

// ---- mbarrier + bulk (TMA) copies into shared memory

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes initialised barriers visible to the async proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk
// copies into shared memory (generic -> async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// ---- L2 cache policies: data that random reads will come back to is kept
// (evict_last), data streamed once goes first (evict_first).

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ ulonglong2 ld_u64x2_hint(const void *a, uint64_t pol) {
    ulonglong2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(v.x), "=l"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ int2 ld_i32x2_hint(const void *a, uint64_t pol) {
    int2 v;
    asm volatile("ld.global.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_i32_hint(void *a, int32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}

// Monotonic nanosecond clock shared by all SMs.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every inter-block wait gives up after this long and reports LOR_ERR_TIMEOUT.
constexpr uint64_t kSpinLimitNs = 2000000000ull;  // 2 s

// The wait limit in force, one copy per translation unit (kSpinLimitNs unless
// lor_test_set_wait changed it), and the test switch that keeps the first
// tile of a radix pass from publishing its look-back descriptor, so that the
// tiles after it must give up waiting on it.
static __device__ uint64_t g_wait_limit_ns = kSpinLimitNs;
static __device__ int g_starve_first_tile = 0;
__device__ __forceinline__ uint64_t wait_limit_ns() { return *(volatile uint64_t *)&g_wait_limit_ns; }

// Waits for phase `parity` of a barrier for at most `limit` ns; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit) return false;
    return true;
}

// Double-buffered bulk loads for a grid-stride loop over tiles of kN
// elements of two arrays: while a block works on one tile, the next tile of
// its stride is on its way into the other buffer.  A whole tile with 16-byte
// aligned rows is copied in bulk; a partial or unaligned one is read from
// global memory by the caller (whole() says which).  Thread 0 issues; every
// thread waits, for at most the wait limit.
template <typename A, typename B, int kN>
struct BulkPair {
    A a[2][kN];
    B b[2][kN];
    uint64_t bar[2];
};

template <typename A, typename B, int kN>
struct BulkPairLoader {
    BulkPair<A, B, kN> &S;
    const A *ga;
    const B *gb;
    int64_t n;
    uint32_t phase;
    __device__ __forceinline__ BulkPairLoader(BulkPair<A, B, kN> &s, const A *a, const B *b, int64_t count)
        : S(s), ga(a), gb(b), n(count), phase(0) {
        if (threadIdx.x == 0) {
            mbar_init(&S.bar[0], 1);
            mbar_init(&S.bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    __device__ __forceinline__ bool whole(int64_t t) const {
        return t >= 0 && (t + 1) * kN <= n && (uintptr_t(ga + t * kN) & 15) == 0 &&
               (uintptr_t(gb + t * kN) & 15) == 0;
    }
    // thread 0: start the copy of tile t into buffer buf (after the buffer's
    // last readers passed a barrier)
    __device__ __forceinline__ void issue(int64_t t, int buf) {
        if (!whole(t)) return;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&S.bar[buf], uint32_t(kN * (sizeof(A) + sizeof(B))));
        bulk_g2s(S.a[buf], ga + t * kN, uint32_t(kN * sizeof(A)), &S.bar[buf]);
        bulk_g2s(S.b[buf], gb + t * kN, uint32_t(kN * sizeof(B)), &S.bar[buf]);
    }
    // every thread: wait for tile t in buffer buf; false when the wait ran out
    __device__ __forceinline__ bool wait(int64_t t, int buf, uint64_t limit) {
        if (!whole(t)) return true;
        const bool ok = mbar_wait_bounded(&S.bar[buf], (phase >> buf) & 1u, limit);
        phase ^= 1u << buf;
        return ok;
    }
    // thread 0, on the way out after a wait ran out: give the copies still in
    // flight a bounded time to land
    __device__ __forceinline__ void drain(int64_t t, int buf, int64_t nxt, uint64_t limit) {
        if (whole(t)) mbar_wait_bounded(&S.bar[buf], ((phase >> buf) & 1u) ^ 1u, limit);
        if (whole(nxt)) mbar_wait_bounded(&S.bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, limit);
    }
};

// The same for one array.
template <typename A, int kN>
struct BulkOne {
    A a[2][kN];
    uint64_t bar[2];
};

template <typename A, int kN>
struct BulkOneLoader {
    BulkOne<A, kN> &S;
    const A *ga;
    int64_t n;
    uint32_t phase;
    __device__ __forceinline__ BulkOneLoader(BulkOne<A, kN> &s, const A *a, int64_t count)
        : S(s), ga(a), n(count), phase(0) {
        if (threadIdx.x == 0) {
            mbar_init(&S.bar[0], 1);
            mbar_init(&S.bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    __device__ __forceinline__ bool whole(int64_t t) const {
        return t >= 0 && (t + 1) * kN <= n && (uintptr_t(ga + t * kN) & 15) == 0;
    }
    __device__ __forceinline__ void issue(int64_t t, int buf) {
        if (!whole(t)) return;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&S.bar[buf], uint32_t(kN * sizeof(A)));
        bulk_g2s(S.a[buf], ga + t * kN, uint32_t(kN * sizeof(A)), &S.bar[buf]);
    }
    __device__ __forceinline__ bool wait(int64_t t, int buf, uint64_t limit) {
        if (!whole(t)) return true;
        const bool ok = mbar_wait_bounded(&S.bar[buf], (phase >> buf) & 1u, limit);
        phase ^= 1u << buf;
        return ok;
    }
    __device__ __forceinline__ void drain(int64_t t, int buf, int64_t nxt, uint64_t limit) {
        if (whole(t)) mbar_wait_bounded(&S.bar[buf], ((phase >> buf) & 1u) ^ 1u, limit);
        if (whole(nxt)) mbar_wait_bounded(&S.bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, limit);
    }
};

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Decoupled look-back descriptors: [epoch:30 | flag:2 | value:32].
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;
__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint64_t flag, uint32_t v) {
    return (uint64_t(epoch) << 34) | (flag << 32) | uint64_t(v);
}
__device__ __forceinline__ uint32_t lb_epoch(uint64_t w) { return uint32_t(w >> 34); }
__device__ __forceinline__ uint32_t lb_flag(uint64_t w) { return uint32_t((w >> 32) & 3); }
__device__ __forceinline__ uint32_t lb_value(uint64_t w) { return uint32_t(w); }

// Inclusive warp scan of 32-bit values.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x = NT, multiple of
// 32, at most 1024).  `scratch` needs NT/32 + 1 words.  Returns the exclusive
// prefix; *total receives the block sum.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *scratch, uint32_t *total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? scratch[lane] : 0;
        uint32_t wi = warp_incl_scan(w);
        if (lane < NW) scratch[lane] = wi - w;
        if (lane == NW - 1) scratch[NW] = wi;
    }
    __syncthreads();
    uint32_t excl = scratch[warp] + inc - v;
    *total = scratch[NW];
    __syncthreads();
    return excl;
}

// Single-value decoupled look-back performed by warp 0 of a block: publishes
// the tile aggregate, walks back over predecessors 32 at a time, publishes
// the inclusive prefix and returns the exclusive prefix (to lane 0..31).
// Every wait is bounded; on expiry *status gets LOR_ERR_TIMEOUT.
__device__ __forceinline__ uint32_t warp_lookback(uint64_t *lb, int64_t tile, uint32_t agg,
                                                  uint32_t epoch, int *status) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_volatile_u64(&lb[0], lb_pack(epoch, kFlagIncl, agg));
        return 0;
    }
    if (lane == 0) st_volatile_u64(&lb[tile], lb_pack(epoch, kFlagAgg, agg));
    uint32_t excl = 0;
    int64_t j = tile - 1;
    const uint64_t t0 = global_ns(), limit = wait_limit_ns();
    bool timed_out = false;
    while (true) {
        int64_t idx = j - lane;
        uint64_t w = idx >= 0 ? ld_volatile_u64(&lb[idx]) : lb_pack(epoch, kFlagIncl, 0);
        while (true) {
            bool ready = lb_epoch(w) == epoch && lb_flag(w) != 0;
            if (__all_sync(0xffffffffu, ready)) break;
            if (!ready) w = ld_volatile_u64(&lb[idx]);
            // warp-uniform decision: every lane leaves the loop together
            if (__any_sync(0xffffffffu, global_ns() - t0 > limit)) { timed_out = true; break; }
        }
        if (timed_out) {
            if (lane == 0) atomicCAS(status, 0, LOR_ERR_TIMEOUT);
            break;
        }
        uint32_t incl_mask = __ballot_sync(0xffffffffu, lb_flag(w) == kFlagIncl);
        uint32_t v = lb_value(w);
        if (incl_mask) {
            int first = __ffs(incl_mask) - 1;
            v = lane <= first ? v : 0;
            excl += warp_sum(v);
            break;
        }
        excl += warp_sum(v);
        j -= 32;
    }
    if (lane == 0) {
        __threadfence();
        st_volatile_u64(&lb[tile], lb_pack(epoch, kFlagIncl, excl + agg));
    }
    return excl;
}

}  // namespace lor

namespace lor {
// A status slot that replaces the translation units' status words for the
// launches of the calling host thread (nullptr: the words are used).  Server
// workers point it at a slot of their own, so that their batches neither see
// nor clear each other's errors.
int *status_slot();
void set_status_slot(int *d_slot);
// Reads the slot after the stream's work, clears it when set, returns it.
int read_status_slot(int *d_slot, cudaStream_t s);
}  // namespace lor

// One device status word per translation unit; kernels record the first
// error with atomicCAS and the host reads it through the TU's accessor.  The
// TU's wait limit and starve switch are set through name##_set_wait.
#define LOR_DEFINE_TU_STATUS(name)                                                    \
    static __device__ int g_tu_status;                                                \
    int name##_set_wait(uint64_t limit_ns, int starve) {                              \
        if (cudaMemcpyToSymbol(lor::g_wait_limit_ns, &limit_ns, sizeof(limit_ns)) !=       \
                cudaSuccess ||                                                        \
            cudaMemcpyToSymbol(lor::g_starve_first_tile, &starve, sizeof(starve)) !=       \
                cudaSuccess)                                                          \
            return LOR_ERR_CUDA;                                                      \
        return LOR_OK;                                                                \
    }                                                                                 \
    int name(cudaStream_t s, int clear) {                                             \
        int h = 0;                                                                    \
        if (cudaMemcpyFromSymbolAsync(&h, g_tu_status, sizeof(int), 0,               \
                                      cudaMemcpyDeviceToHost, s) != cudaSuccess)      \
            return LOR_ERR_CUDA;                                                      \
        if (cudaStreamSynchronize(s) != cudaSuccess) return LOR_ERR_CUDA;             \
        if (clear && h != 0) {                                                        \
            int z = 0;                                                                \
            if (cudaMemcpyToSymbolAsync(g_tu_status, &z, sizeof(int), 0,              \
                                        cudaMemcpyHostToDevice, s) != cudaSuccess)    \
                return LOR_ERR_CUDA;                                                  \
            if (cudaStreamSynchronize(s) != cudaSuccess) return LOR_ERR_CUDA;         \
        }                                                                             \
        return h;                                                                     \
    }                                                                                 \
    static int *tu_status_ptr() {                                                     \
        if (int *o = lor::status_slot()) return o;                                    \
        static thread_local int *p = nullptr;                                         \
        static thread_local int dev = -1;                                             \
        int cur = -1;                                                                 \
        cudaGetDevice(&cur);                                                          \
        if (p == nullptr || dev != cur) {                                             \
            void *q = nullptr;                                                        \
            if (cudaGetSymbolAddress(&q, g_tu_status) != cudaSuccess) return nullptr; \
            p = (int *)q;                                                             \
            dev = cur;                                                                \
        }                                                                             \
        return p;                                                                     \
    }

// Accessors of every translation unit's status word (one per .cu file).
int lor_status_encode(cudaStream_t s, int clear);
int lor_status_dc3(cudaStream_t s, int clear);
int lor_status_lcp(cudaStream_t s, int clear);
int lor_status_overlap(cudaStream_t s, int clear);
int lor_status_rmq(cudaStream_t s, int clear);
int lor_status_abi(cudaStream_t s, int clear);
int lor_status_batch(cudaStream_t s, int clear);
int lor_status_serve(cudaStream_t s, int clear);
int lor_status_multi(cudaStream_t s, int clear);
int lor_status_topk(cudaStream_t s, int clear);
int lor_status_sa64(cudaStream_t s, int clear);
int lor_status_encode_set_wait(uint64_t limit_ns, int starve);
int lor_status_dc3_set_wait(uint64_t limit_ns, int starve);
int lor_status_lcp_set_wait(uint64_t limit_ns, int starve);
int lor_status_overlap_set_wait(uint64_t limit_ns, int starve);
int lor_status_rmq_set_wait(uint64_t limit_ns, int starve);
int lor_status_abi_set_wait(uint64_t limit_ns, int starve);
int lor_status_batch_set_wait(uint64_t limit_ns, int starve);
int lor_status_serve_set_wait(uint64_t limit_ns, int starve);
int lor_status_multi_set_wait(uint64_t limit_ns, int starve);
int lor_status_topk_set_wait(uint64_t limit_ns, int starve);
int lor_status_sa64_set_wait(uint64_t limit_ns, int starve);

namespace lor {
// Sparse-table rows 0..levels-1 over lcp[0..n) (rmq.cu); rows are
// row_stride(n) = n rounded up to 64 entries apart, table 256-byte aligned.
int rmq_build_levels(const int32_t *d_lcp, int64_t n, int levels, int32_t *d_table, cudaStream_t s);
}  // namespace lor
