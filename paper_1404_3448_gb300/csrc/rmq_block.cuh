// rmq_block.cuh -- the range minimum of the linear-space (block) RMQ, shared
// by the block-RMQ entry points (rmq.cu) and the request server's resident
// query state (serve.cu).
//
// The LCP array is cut into blocks of kRmqBlock entries and a sparse table is
// kept over the block minima (row j at table + j * stride: minima of windows
// of 2^j blocks).  min(lcp[a .. b]) is the minimum of the partial blocks at
// both ends, scanned in the LCP array, and of the whole blocks between them,
// read from two windows of the table (Section 3: the LCP of two suffixes is
// the minimum of the adjacent LCPs between their ranks).
#pragma once

#include "common.cuh"

namespace lor {

constexpr int kRmqBlock = 32;

__host__ __device__ inline int64_t rmqb_blocks(int64_t n) { return (n + kRmqBlock - 1) / kRmqBlock; }

// min(lcp[a .. b]) for a <= b inside one block.
__device__ __forceinline__ int32_t rmqb_scan(const int32_t *__restrict__ lcp, int64_t a, int64_t b) {
    int32_t m = lcp[a];
    for (int64_t i = a + 1; i <= b; ++i) m = min(m, lcp[i]);
    return m;
}

// min(lcp[a .. b]) for a <= b.
__device__ __forceinline__ int32_t rmqb_range_min(const int32_t *__restrict__ table, int64_t stride,
                                                  const int32_t *__restrict__ lcp, int64_t a, int64_t b) {
    const int64_t ba = a / kRmqBlock, bb = b / kRmqBlock;
    if (ba == bb) return rmqb_scan(lcp, a, b);
    int32_t m = min(rmqb_scan(lcp, a, ba * kRmqBlock + kRmqBlock - 1), rmqb_scan(lcp, bb * kRmqBlock, b));
    const int64_t len = bb - ba - 1;  // whole blocks ba+1 .. bb-1
    if (len > 0) {
        const int j = 63 - __clzll(len);
        const int32_t *lv = table + int64_t(j) * stride;
        m = min(m, min(lv[ba + 1], lv[bb - (int64_t(1) << j)]));
    }
    return m;
}

// The block table over lcp[0..n): `levels` rows of stride rmq_row_stride_of(nb)
// (rmq.cu).
int rmq_block_levels(const int32_t *d_lcp, int64_t n, int levels, int32_t *d_table, cudaStream_t s);
int64_t rmq_row_stride_of(int64_t m);

}  // namespace lor
