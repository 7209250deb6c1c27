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
#include "lcp_kernels.cuh"

LOR_DEFINE_TU_STATUS(lor_status_lcp)

namespace lor {
namespace {

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
        k_isa_phi<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, nullptr, ip, status);
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
