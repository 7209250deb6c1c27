// rmq.cu -- sparse table over the LCP array and LCP queries between arbitrary
// suffixes (Section 3: the LCP of two suffixes is the minimum of the adjacent
// LCPs between their ranks; RMQ returns that minimum in O(1) per query).
//
// Level j holds the minimum of every window of 2^j entries (clipped at the
// end of the array): table[j][i] = min(table[j-1][i], table[j-1][i + 2^(j-1)]).
// A query over ranks (r1, r2] reads two overlapping windows of level
// floor(log2(r2 - r1)).
#include "common.cuh"

LOR_DEFINE_TU_STATUS(lor_status_rmq)

namespace lor {
namespace {

int levels_for(int64_t n) { return n > 0 ? bit_width_u64(uint64_t(n)) : 1; }

__global__ void k_copy_i32(const int32_t *__restrict__ src, int32_t *__restrict__ dst, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

__global__ void k_rmq_level(const int32_t *__restrict__ src, int32_t *__restrict__ dst, int64_t n,
                            int64_t h) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = src[i];
    dst[i] = (i + h < n) ? min(a, src[i + h]) : a;
}

__global__ void k_rmq_query(const int32_t *__restrict__ table, const int32_t *__restrict__ isa,
                            int64_t n, const int32_t *__restrict__ P, const int32_t *__restrict__ Q,
                            int64_t nq, int32_t *__restrict__ out, int *status) {
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
    const int32_t *lv = table + int64_t(j) * n;
    out[i] = min(lv[r1 + 1], lv[r2 - (int64_t(1) << j) + 1]);
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" int64_t lor_rmq_table_elems(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return int64_t(levels_for(n)) * n;
}

extern "C" int lor_rmq_build(const int32_t *d_lcp, int64_t n, int32_t *d_table, int64_t table_elems,
                             lor_stream_t stream) {
    if (!d_lcp || !d_table || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    if (table_elems < lor_rmq_table_elems(n)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = unsigned(cdiv(n, 256));
    {
        ProfScope ps(PK_RMQ_LEVEL, double(n) * 8, s);
        k_copy_i32<<<grid, 256, 0, s>>>(d_lcp, d_table, n);
    }
    LOR_LAUNCH_CHECK();
    const int J = levels_for(n);
    for (int j = 1; j < J; ++j) {
        ProfScope ps(PK_RMQ_LEVEL, double(n) * 8, s);
        k_rmq_level<<<grid, 256, 0, s>>>(d_table + int64_t(j - 1) * n, d_table + int64_t(j) * n, n,
                                         int64_t(1) << (j - 1));
        LOR_LAUNCH_CHECK();
    }
    return LOR_OK;
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
        k_rmq_query<<<unsigned(cdiv(nq, 256)), 256, 0, s>>>(d_table, d_isa, n, d_p, d_q, nq, d_out,
                                                            status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
