// lcp.cu -- inverse suffix array and LCP array (Section 3, LCP table; the
// linear-time method of Kasai et al. that the paper cites).
//
// Kasai's observation: for text positions i and i+1, the LCP of suffix i+1
// with its rank predecessor is at least the LCP of suffix i with its rank
// predecessor minus one.  It is applied here in the "permuted LCP" form:
//   1. one scatter per rank k writes {ISA, PHI} = {k, SA[k-1]} at position
//      SA[k] (one 8-byte write instead of separate ISA / predecessor lookups);
//   2. text positions are walked in order in chunks (h carried within a
//      chunk), comparing T[i+h..] with T[PHI[i]+h..] four bytes at a time, and
//      PLCP[i] and ISA[i] are written in text order;
//   3. LCP[k] = PLCP[SA[k]] is gathered in rank order.
#include "common.cuh"

LOR_DEFINE_TU_STATUS(lor_status_lcp)

namespace lor {
namespace {

__global__ void k_isa_phi(const int32_t *__restrict__ sa, int64_t n, int2 *__restrict__ ip, int *status) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    if (p < 0 || p >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    ip[p] = make_int2(int32_t(k), k > 0 ? sa[k - 1] : -1);
}

// Four text bytes starting at byte offset a (little-endian), from two aligned
// words; the caller guarantees a + 8 <= n.
__device__ __forceinline__ uint32_t load4(const uint8_t *t, int64_t a) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(t + (a & ~int64_t(3)));
    return __funnelshift_r(w[0], w[1], uint32_t(a & 3) * 8u);
}

constexpr int kPlcpThreads = 256;
constexpr int kPlcpPer = 16;  // text positions per thread
constexpr int kPlcpTile = kPlcpThreads * kPlcpPer;

__global__ void __launch_bounds__(kPlcpThreads) k_plcp(const uint8_t *__restrict__ t, int64_t n,
                                                       const int2 *__restrict__ ip,
                                                       int32_t *__restrict__ isa, int32_t *__restrict__ plcp,
                                                       int aligned, int *status) {
    __shared__ int2 s_ip[kPlcpTile];
    __shared__ int32_t s_out[kPlcpTile];
    const int64_t base = int64_t(blockIdx.x) * kPlcpTile;
    const int cnt = int(min64(int64_t(kPlcpTile), n - base));
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) {
        const int2 v = ip[base + i];
        s_ip[i] = v;
        isa[base + i] = v.x;
    }
    __syncthreads();
    int64_t h = 0;
    bool bad = false;
    const int l0 = int(threadIdx.x) * kPlcpPer;
    for (int l = l0; l < l0 + kPlcpPer && l < cnt; ++l) {
        const int64_t i = base + l;
        const int64_t j = s_ip[l].y;
        if (j < 0 || j >= n) {
            if (j != -1) bad = true;
            h = 0;
            s_out[l] = 0;
            continue;
        }
        bool found = false;
        if (aligned) {
            while (i + h + 8 <= n && j + h + 8 <= n) {
                const uint32_t x = load4(t, i + h) ^ load4(t, j + h);
                if (x) {
                    h += (__ffs(x) - 1) >> 3;  // equal low-order (leading) bytes
                    found = true;
                    break;
                }
                h += 4;
            }
        }
        if (!found)
            while (i + h < n && j + h < n && t[i + h] == t[j + h]) ++h;
        s_out[l] = int32_t(h);
        if (h > 0) --h;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) plcp[base + i] = s_out[i];
}

__global__ void k_lcp_gather(const int32_t *__restrict__ sa, int64_t n, const int32_t *__restrict__ plcp,
                             int32_t *__restrict__ lcp) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    lcp[k] = (k == 0 || p < 0 || p >= n) ? 0 : plcp[p];
}

struct LcpLayout {
    size_t ip = 0, plcp = 0, total = 0;
};
LcpLayout lcp_layout(int64_t n) {
    LcpLayout L;
    L.ip = 0;
    L.plcp = align256(sizeof(int2) * size_t(n));
    L.total = L.plcp + align256(sizeof(int32_t) * size_t(n));
    return L;
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_lcp_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N) return 0;
    return lcp_layout(n).total;
}

extern "C" int lor_lcp(const uint8_t *d_text, const int32_t *d_sa, int64_t n, int32_t *d_isa,
                       int32_t *d_lcp, void *d_ws, size_t ws_bytes, lor_stream_t stream) {
    if (!d_text || !d_sa || !d_isa || !d_lcp || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const LcpLayout L = lcp_layout(n);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    int2 *ip = (int2 *)((char *)d_ws + L.ip);
    int32_t *plcp = (int32_t *)((char *)d_ws + L.plcp);
    {
        // SA read (4 + 4 neighbour), 8-byte scatter
        ProfScope ps(PK_ISA_SCATTER, double(n) * 12, s);
        k_isa_phi<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, ip, status);
    }
    LOR_LAUNCH_CHECK();
    {
        // {ISA, PHI} read, ISA + PLCP written, two text reads per position
        ProfScope ps(PK_KASAI, double(n) * (8 + 4 + 4 + 2), s);
        const int aligned = (uintptr_t(d_text) & 3) == 0;
        k_plcp<<<unsigned(cdiv(n, kPlcpTile)), kPlcpThreads, 0, s>>>(d_text, n, ip, d_isa, plcp, aligned,
                                                                     status);
    }
    LOR_LAUNCH_CHECK();
    {
        ProfScope ps(PK_KASAI, double(n) * 12, s);
        k_lcp_gather<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, plcp, d_lcp);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}
