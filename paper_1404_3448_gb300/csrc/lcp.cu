// lcp.cu -- inverse suffix array and LCP array (Section 3, LCP table; the
// linear-time method of Kasai et al. that the paper cites).
//
// Kasai's observation: for text positions i and i+1, lcp at rank ISA[i+1] is
// at least lcp at rank ISA[i] minus one.  Each thread walks one contiguous
// chunk of text positions carrying h across the chunk (starting from 0 at its
// first position), so total symbol comparisons stay linear plus one
// from-scratch comparison per chunk.
#include "common.cuh"

LOR_DEFINE_TU_STATUS(lor_status_lcp)

namespace lor {
namespace {

__global__ void k_isa_scatter(const int32_t *__restrict__ sa, int64_t n, int32_t *__restrict__ isa,
                              int *status) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    if (p < 0 || p >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    isa[p] = int32_t(k);
}

constexpr int kKasaiChunk = 64;

__global__ void __launch_bounds__(256) k_kasai(const uint8_t *__restrict__ t, const int32_t *__restrict__ sa,
                                               const int32_t *__restrict__ isa, int64_t n,
                                               int32_t *__restrict__ lcp, int *status) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t i0 = g * kKasaiChunk;
    if (i0 >= n) return;
    const int64_t i1 = i0 + kKasaiChunk < n ? i0 + kKasaiChunk : n;
    int64_t h = 0;
    for (int64_t i = i0; i < i1; ++i) {
        const int32_t r = isa[i];
        if (r < 0 || r >= n) {
            atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
            h = 0;
            continue;
        }
        if (r == 0) {
            lcp[0] = 0;
            h = 0;
            continue;
        }
        const int32_t j = sa[r - 1];
        if (j < 0 || j >= n) {
            atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
            h = 0;
            continue;
        }
        while (i + h < n && j + h < n && t[i + h] == t[j + h]) ++h;
        lcp[r] = int32_t(h);
        if (h > 0) --h;
    }
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" int lor_lcp(const uint8_t *d_text, const int32_t *d_sa, int64_t n, int32_t *d_isa,
                       int32_t *d_lcp, lor_stream_t stream) {
    if (!d_text || !d_sa || !d_isa || !d_lcp || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    {
        ProfScope ps(PK_ISA_SCATTER, double(n) * 8, s);
        k_isa_scatter<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, d_isa, status);
    }
    LOR_LAUNCH_CHECK();
    {
        // ISA read, SA gather, two text reads, LCP write per position
        ProfScope ps(PK_KASAI, double(n) * (4 + 4 + 2 + 4), s);
        k_kasai<<<unsigned(cdiv(cdiv(n, kKasaiChunk), 256)), 256, 0, s>>>(d_text, d_sa, d_isa, n, d_lcp,
                                                                          status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
