// rmq.cu -- sparse table over the LCP array and LCP queries between arbitrary
// suffixes (Section 3: the LCP of two suffixes is the minimum of the adjacent
// LCPs between their ranks; RMQ returns that minimum in O(1) per query).
//
// Level j holds the minimum of every window of 2^j entries (clipped at the
// end of the array): table[j][i] = min(table[j-1][i], table[j-1][i + 2^(j-1)]).
// Rows are padded to a multiple of 64 entries so that every row starts on a
// 256-byte boundary.  Levels 0..8 are produced by one kernel that stages a
// tile plus a 256-entry halo of the LCP array in shared memory and writes the
// nine rows; the higher levels are made three at a time by comb passes with
// 16-byte accesses (k_rmq_comb; the operands, multiples of 2^(j-1) >= 256
// entries apart, are 16-byte aligned too).
// A query over ranks (r1, r2] reads two overlapping windows of level
// floor(log2(r2 - r1)).
#include <climits>

#include "rmq_block.cuh"

LOR_DEFINE_TU_STATUS(lor_status_rmq)

namespace lor {
namespace {

int levels_for(int64_t n) { return n > 0 ? bit_width_u64(uint64_t(n)) : 1; }
int64_t row_stride(int64_t n) { return (n + 63) & ~int64_t(63); }

constexpr int kLowLevels = 8;               // levels 1..8 from shared memory
constexpr int kLowHalo = 1 << kLowLevels;   // 256 >= 2^8 - 1
constexpr int kLowTile = 4096;
constexpr int kLowThreads = 256;
constexpr int kLowPer = (kLowTile + kLowHalo) / kLowThreads;  // 17

__global__ void __launch_bounds__(kLowThreads) k_rmq_low(const int32_t *__restrict__ lcp, int64_t n,
                                                         int32_t *__restrict__ table, int64_t stride,
                                                         int top) {
    __shared__ int32_t buf[kLowTile + kLowHalo];
    const int64_t base = int64_t(blockIdx.x) * kLowTile;
    const int tid = threadIdx.x;
    int32_t v[kLowPer];
#pragma unroll
    for (int k = 0; k < kLowPer; ++k) {
        const int64_t i = base + tid + k * kLowThreads;
        v[k] = i < n ? lcp[i] : INT_MAX;  // clipped windows: padding never wins
        buf[tid + k * kLowThreads] = v[k];
    }
    const int out_n = int(min64(int64_t(kLowTile), n - base));
#pragma unroll
    for (int k = 0; k < kLowPer; ++k) {
        const int i = tid + k * kLowThreads;
        if (i < out_n) table[base + i] = v[k];
    }
    for (int j = 1; j <= top; ++j) {
        const int h = 1 << (j - 1);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kLowPer; ++k) {
            const int i = tid + k * kLowThreads;
            if (i + h < kLowTile + kLowHalo) v[k] = min(v[k], buf[i + h]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kLowPer; ++k) buf[tid + k * kLowThreads] = v[k];
        int32_t *row = table + int64_t(j) * stride + base;
#pragma unroll
        for (int k = 0; k < kLowPer; ++k) {
            const int i = tid + k * kLowThreads;
            if (i < out_n) row[i] = v[k];
        }
    }
}

// K levels per pass over a comb: a thread loads the 16-byte groups at
// x0 + q*h (q = 0 .. Q + 2^K - 2) of level j-1 (windows of h = 2^(j-1)) once,
// and writes levels j .. j+K-1 at x0 + q*h (q < Q) from them: level j+k at a
// position is the minimum of the 2^(k+1) level-(j-1) windows h apart that
// start there, computed in place by doubling.  A row is read about
// (Q + 2^K - 1) / Q times per pass whatever h is, where a pass that reads
// its operands in address order re-reads far operands from DRAM once h
// outgrows the L2.  Entries past n read as INT_MAX (windows are clipped).
__device__ __forceinline__ int4 rmq_load4(const int32_t *__restrict__ src, int64_t x, int64_t n) {
    if (x + 3 < n) return *reinterpret_cast<const int4 *>(src + x);
    int4 r;
    r.x = x + 0 < n ? src[x + 0] : INT_MAX;
    r.y = x + 1 < n ? src[x + 1] : INT_MAX;
    r.z = x + 2 < n ? src[x + 2] : INT_MAX;
    r.w = x + 3 < n ? src[x + 3] : INT_MAX;
    return r;
}

__device__ __forceinline__ int4 min4(int4 a, int4 b) {
    return make_int4(min(a.x, b.x), min(a.y, b.y), min(a.z, b.z), min(a.w, b.w));
}

template <int K, int Q>
__global__ void __launch_bounds__(256) k_rmq_comb(const int32_t *__restrict__ src, int32_t *__restrict__ dst,
                                                  int64_t stride, int64_t n, int64_t h) {
    constexpr int W = 1 << K;
    constexpr int L = Q + W - 1;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t hq = h / 4;  // 16-byte groups per h entries (h is a multiple of 4)
    const int64_t g = t / hq;
    const int64_t x0 = g * Q * h + (t - g * hq) * 4;
    if (x0 >= n) return;
    int4 s[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const int64_t x = x0 + int64_t(q) * h;
        s[q] = x < n ? rmq_load4(src, x, n) : make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int d = 1 << k;
#pragma unroll
        for (int q = 0; q + d < L; ++q) s[q] = min4(s[q], s[q + d]);
        int32_t *row = dst + int64_t(k) * stride;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t x = x0 + int64_t(q) * h;
            if (x < n) *reinterpret_cast<int4 *>(row + x) = s[q];  // rows are padded to 64 entries
        }
    }
}

__global__ void k_rmq_query(const int32_t *__restrict__ table, int64_t stride,
                            const int32_t *__restrict__ isa, int64_t n, const int32_t *__restrict__ P,
                            const int32_t *__restrict__ Q, int64_t nq, int32_t *__restrict__ out,
                            int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const int32_t p = P[i], q = Q[i];
    if (p < 0 || p >= n || q < 0 || q >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    if (p == q) {
        out[i] = int32_t(n - p);
        return;
    }
    int32_t r1 = isa[p], r2 = isa[q];
    if (r1 < 0 || r1 >= n || r2 < 0 || r2 >= n || r1 == r2) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    if (r1 > r2) {
        const int32_t tmp = r1;
        r1 = r2;
        r2 = tmp;
    }
    const int64_t len = int64_t(r2) - r1;  // window (r1, r2] of len entries
    const int j = 63 - __clzll(len);
    const int32_t *lv = table + int64_t(j) * stride;
    out[i] = min(lv[r1 + 1], lv[r2 - (int64_t(1) << j) + 1]);
}

// ---- block-sparse RMQ in linear space
//
// The LCP array is cut into blocks of kRmqBlock entries; a sparse table is
// built over the block minima only (n / 32 entries per row instead of n), and
// a query over ranks (r1, r2] takes the minimum of the partial blocks at both
// ends, read from the LCP array itself, and of the whole blocks between them,
// read from two windows of the block table.


// bm[b] = min(lcp[32b .. min(32b + 32, n) - 1]): one warp per block.
__global__ void k_rmqb_blockmin(const int32_t *__restrict__ lcp, int64_t n, int64_t nb, int32_t *__restrict__ bm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t b = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        const int64_t i = b * kRmqBlock + lane;
        const int v = i < n ? lcp[i] : INT_MAX;
        const int m = __reduce_min_sync(0xffffffffu, v);
        if (lane == 0) bm[b] = m;
    }
}


// IdxT: int32 or int64 ISA and query positions; OutT: int32 or int64 answers
// (p == q answers the suffix length n - p, which needs 64 bits past 2^31).
template <typename IdxT, typename OutT>
__global__ void k_rmqb_query(const int32_t *__restrict__ table, int64_t stride, const int32_t *__restrict__ lcp,
                             const IdxT *__restrict__ isa, int64_t n, const IdxT *__restrict__ P,
                             const IdxT *__restrict__ Q, int64_t nq, OutT *__restrict__ out, int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const int64_t p = P[i], q = Q[i];
    if (p < 0 || p >= n || q < 0 || q >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    if (p == q) {
        out[i] = OutT(n - p);
        return;
    }
    int64_t r1 = isa[p], r2 = isa[q];
    if (r1 < 0 || r1 >= n || r2 < 0 || r2 >= n || r1 == r2) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    if (r1 > r2) {
        const int64_t tmp = r1;
        r1 = r2;
        r2 = tmp;
    }
    out[i] = OutT(rmqb_range_min(table, stride, lcp, r1 + 1, r2));
}

// First index in [a, b] (one block) holding the value v, or -1.
__device__ __forceinline__ int64_t rmqb_first(const int32_t *__restrict__ lcp, int64_t a, int64_t b, int32_t v) {
    for (int64_t i = a; i <= b; ++i)
        if (lcp[i] == v) return i;
    return -1;
}

// The leftmost minimum of lcp(r1, r2] (Section 3: the RMQ returns the index
// of the minimum; the leftmost one when it repeats) and its value.  After the
// value m is known, the partial block at the left end is scanned first; then
// the leftmost whole block whose minimum is m is found by binary lifting over
// the table rows (skip every power-of-two window, largest first, whose
// minimum exceeds m) and scanned; last the partial block at the right end.
__global__ void k_rmqb_argmin(const int32_t *__restrict__ table, int64_t stride, const int32_t *__restrict__ lcp,
                              const int32_t *__restrict__ isa, int64_t n, const int32_t *__restrict__ P,
                              const int32_t *__restrict__ Q, int64_t nq, int32_t *__restrict__ val,
                              int32_t *__restrict__ arg, int *status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const int32_t p = P[i], q = Q[i];
    if (p < 0 || p >= n || q < 0 || q >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        val[i] = -1;
        arg[i] = -1;
        return;
    }
    if (p == q) {
        val[i] = int32_t(n - p);
        arg[i] = -1;
        return;
    }
    int32_t r1 = isa[p], r2 = isa[q];
    if (r1 < 0 || r1 >= n || r2 < 0 || r2 >= n || r1 == r2) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        val[i] = -1;
        arg[i] = -1;
        return;
    }
    if (r1 > r2) {
        const int32_t tmp = r1;
        r1 = r2;
        r2 = tmp;
    }
    const int64_t a = int64_t(r1) + 1, b = r2;
    const int64_t ba = a / kRmqBlock, bb = b / kRmqBlock;
    int32_t m;
    int64_t k;
    if (ba == bb) {
        m = rmqb_scan(lcp, a, b);
        k = rmqb_first(lcp, a, b, m);
    } else {
        const int64_t aend = ba * kRmqBlock + kRmqBlock - 1, bbeg = bb * kRmqBlock;
        const int32_t ma = rmqb_scan(lcp, a, aend), mb = rmqb_scan(lcp, bbeg, b);
        m = min(ma, mb);
        const int64_t lo = ba + 1, hi = bb - 1;  // whole blocks
        int32_t mw = INT_MAX;
        if (hi >= lo) {
            const int j = 63 - __clzll(hi - lo + 1);
            const int32_t *lv = table + int64_t(j) * stride;
            mw = min(lv[lo], lv[hi - (int64_t(1) << j) + 1]);
            m = min(m, mw);
        }
        if (ma == m) {
            k = rmqb_first(lcp, a, aend, m);
        } else if (mw == m) {
            int64_t pos = lo;
            for (int j = 63 - __clzll(hi - lo + 1); j >= 0; --j)
                if (pos + (int64_t(1) << j) - 1 <= hi && table[int64_t(j) * stride + pos] > m) pos += int64_t(1) << j;
            k = rmqb_first(lcp, pos * kRmqBlock, min64(pos * kRmqBlock + kRmqBlock - 1, n - 1), m);
        } else {
            k = rmqb_first(lcp, bbeg, b, m);
        }
    }
    val[i] = m;
    arg[i] = int32_t(k);
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" int lor_rmq_block_argmin(const int32_t *d_table, const int32_t *d_lcp, const int32_t *d_isa, int64_t n,
                                    const int32_t *d_p, const int32_t *d_q, int64_t nq, int32_t *d_val,
                                    int32_t *d_arg, lor_stream_t stream) {
    if (!d_table || !d_lcp || !d_isa || n < 1 || nq < 0) return LOR_ERR_INVALID_ARG;
    if (nq == 0) return LOR_OK;
    if (!d_p || !d_q || !d_val || !d_arg) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    {
        ProfScope ps(PK_RMQ_QUERY, double(nq) * (4 * 10), s);
        k_rmqb_argmin<<<unsigned(cdiv(nq, 256)), 256, 0, s>>>(d_table, row_stride(rmqb_blocks(n)), d_lcp, d_isa, n,
                                                              d_p, d_q, nq, d_val, d_arg, status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

extern "C" int64_t lor_rmq_block_table_elems(int64_t n) {
    if (n < 1 || n > LOR_MAX_N64) return 0;
    const int64_t nb = rmqb_blocks(n);
    return int64_t(levels_for(nb)) * row_stride(nb);
}

int64_t lor::rmq_row_stride_of(int64_t m) { return row_stride(m); }

int lor::rmq_block_levels(const int32_t *d_lcp, int64_t n, int levels, int32_t *d_table, cudaStream_t s) {
    const int64_t nb = rmqb_blocks(n);
    {
        ProfScope ps(PK_RMQ_LEVEL, double(n) * 4 + double(nb) * 4, s);
        const unsigned grid = unsigned(min64(cdiv(nb * 32, 256), 152 * 16));
        k_rmqb_blockmin<<<grid, 256, 0, s>>>(d_lcp, n, nb, d_table);
    }
    LOR_LAUNCH_CHECK();
    // row 0 now holds the block minima: the rows above are its sparse table
    return rmq_build_levels(d_table, nb, levels, d_table, s);
}

extern "C" int lor_rmq_block_build(const int32_t *d_lcp, int64_t n, int32_t *d_table, int64_t table_elems,
                                   lor_stream_t stream) {
    if (!d_lcp || !d_table || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N64) return LOR_ERR_TOO_LARGE;
    if (table_elems < lor_rmq_block_table_elems(n)) return LOR_ERR_WORKSPACE;
    if (uintptr_t(d_table) & 255) return LOR_ERR_INVALID_ARG;
    return rmq_block_levels(d_lcp, n, levels_for(rmqb_blocks(n)), d_table, (cudaStream_t)stream);
}

extern "C" int lor_rmq_block_query(const int32_t *d_table, const int32_t *d_lcp, const int32_t *d_isa, int64_t n,
                                   const int32_t *d_p, const int32_t *d_q, int64_t nq, int32_t *d_out,
                                   lor_stream_t stream) {
    if (!d_table || !d_lcp || !d_isa || n < 1 || nq < 0) return LOR_ERR_INVALID_ARG;
    if (nq == 0) return LOR_OK;
    if (!d_p || !d_q || !d_out) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    {
        ProfScope ps(PK_RMQ_QUERY, double(nq) * (4 + 4 + 4 + 4 + 4 + 4 + 4 + 4), s);
        k_rmqb_query<int32_t, int32_t><<<unsigned(cdiv(nq, 256)), 256, 0, s>>>(d_table, row_stride(rmqb_blocks(n)), d_lcp, d_isa, n,
                                                             d_p, d_q, nq, d_out, status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

extern "C" int64_t lor_rmq_row_stride(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return row_stride(n);
}

extern "C" int64_t lor_rmq_table_elems(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return int64_t(levels_for(n)) * row_stride(n);
}

int lor::rmq_build_levels(const int32_t *d_lcp, int64_t n, int J, int32_t *d_table, cudaStream_t s) {
    if (J < 1 || J > levels_for(n)) return LOR_ERR_INVALID_ARG;
    const int64_t stride = row_stride(n);
    const int top = J - 1 < kLowLevels ? J - 1 : kLowLevels;
    {
        ProfScope ps(PK_RMQ_LEVEL, double(n) * (4 + 4.0 * (top + 1)), s);
        k_rmq_low<<<unsigned(cdiv(n, kLowTile)), kLowThreads, 0, s>>>(d_lcp, n, d_table, stride, top);
    }
    LOR_LAUNCH_CHECK();
    // Levels above the shared-memory ones: three per comb pass (the last
    // pass takes what is left).
    constexpr int kCombQ = 8;
    for (int j = kLowLevels + 1; j < J;) {
        const int K = J - j < 3 ? J - j : 3;
        const int64_t h = int64_t(1) << (j - 1);
        const int64_t threads = cdiv(n, kCombQ * h) * (h / 4);
        const unsigned grid = unsigned(cdiv(threads, 256));
        const int32_t *src = d_table + int64_t(j - 1) * stride;
        int32_t *dst = d_table + int64_t(j) * stride;
        {
            ProfScope ps(PK_RMQ_LEVEL, double(n) * (4 + 4.0 * K), s);
            if (K == 3) k_rmq_comb<3, kCombQ><<<grid, 256, 0, s>>>(src, dst, stride, n, h);
            else if (K == 2) k_rmq_comb<2, kCombQ><<<grid, 256, 0, s>>>(src, dst, stride, n, h);
            else k_rmq_comb<1, kCombQ><<<grid, 256, 0, s>>>(src, dst, stride, n, h);
        }
        LOR_LAUNCH_CHECK();
        j += K;
    }
    return LOR_OK;
}

extern "C" int lor_rmq_build(const int32_t *d_lcp, int64_t n, int32_t *d_table, int64_t table_elems,
                             lor_stream_t stream) {
    if (!d_lcp || !d_table || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    if (table_elems < lor_rmq_table_elems(n)) return LOR_ERR_WORKSPACE;
    if (uintptr_t(d_table) & 255) return LOR_ERR_INVALID_ARG;
    return rmq_build_levels(d_lcp, n, levels_for(n), d_table, (cudaStream_t)stream);
}

extern "C" int lor_rmq_query(const int32_t *d_table, const int32_t *d_isa, int64_t n, const int32_t *d_p,
                             const int32_t *d_q, int64_t nq, int32_t *d_out, lor_stream_t stream) {
    if (!d_table || !d_isa || n < 1 || nq < 0) return LOR_ERR_INVALID_ARG;
    if (nq == 0) return LOR_OK;
    if (!d_p || !d_q || !d_out) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    {
        ProfScope ps(PK_RMQ_QUERY, double(nq) * (4 + 4 + 4 + 4 + 4 + 4 + 4), s);
        k_rmq_query<<<unsigned(cdiv(nq, 256)), 256, 0, s>>>(d_table, row_stride(n), d_isa, n, d_p, d_q,
                                                            nq, d_out, status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

extern "C" int lor_rmq_block_query64(const int32_t *d_table, const int32_t *d_lcp, const int64_t *d_isa, int64_t n,
                                     const int64_t *d_p, const int64_t *d_q, int64_t nq, int64_t *d_out,
                                     lor_stream_t stream) {
    if (!d_table || !d_lcp || !d_isa || n < 1 || nq < 0) return LOR_ERR_INVALID_ARG;
    if (nq == 0) return LOR_OK;
    if (!d_p || !d_q || !d_out) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N64) return LOR_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    {
        ProfScope ps(PK_RMQ_QUERY, double(nq) * (8 + 8 + 8 + 8 + 4 + 4 + 4 + 4 + 8), s);
        k_rmqb_query<int64_t, int64_t><<<unsigned(cdiv(nq, 256)), 256, 0, s>>>(
            d_table, row_stride(rmqb_blocks(n)), d_lcp, d_isa, n, d_p, d_q, nq, d_out, status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
