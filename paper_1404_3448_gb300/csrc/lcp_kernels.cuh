// lcp_kernels.cuh -- the three LCP kernels (Section 3, LCP table; Kasai et
// al., cited there), shared by lor_lcp and the batched pipeline:
//   k_isa_phi   {ISA, PHI} = {k, SA[k-1]} scattered to position SA[k];
//   k_plcp      text positions in order (h carried within a chunk), comparing
//               T[i+h..] with T[PHI[i]+h..] four bytes at a time: ISA and PLCP
//               in text order;
//   k_lcp_gather LCP[k] = PLCP[SA[k]].
#pragma once

#include "common.cuh"

namespace lor {
namespace {

// ip[SA[k]] = {k, SA[k-1]}; with segment keys, the first rank of every
// segment (seg[k] != seg[k-1]) gets no predecessor (-1).
__global__ void k_isa_phi(const int32_t *__restrict__ sa, int64_t n, const uint32_t *__restrict__ seg,
                          int2 *__restrict__ ip, int *status) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    if (p < 0 || p >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    const bool head = k == 0 || (seg && seg[k] != seg[k - 1]);
    ip[p] = make_int2(int32_t(k), head ? -1 : sa[k - 1]);
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

// LCP[k] = PLCP[SA[k]] (a position without predecessor has PLCP 0).
__global__ void k_lcp_gather(const int32_t *__restrict__ sa, int64_t n, const int32_t *__restrict__ plcp,
                             int32_t *__restrict__ lcp) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    lcp[k] = (k == 0 || p < 0 || p >= n) ? 0 : plcp[p];
}

}  // namespace
}  // namespace lor
