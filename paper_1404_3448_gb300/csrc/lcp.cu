// lcp.cu -- inverse suffix array and LCP array (Section 3, LCP table; the
// linear-time method of Kasai et al. that the paper cites).
//
// LCP[k] is first computed in rank order by comparing the suffixes SA[k-1]
// and SA[k] directly on a 2-bit copy of the text (which stays in L2 for
// DNA), up to 64 symbols; the few ranks that reach that are finished up to
// 8192 symbols, and ISA[SA[k]] = k is one bucketed scatter.  This reads and
// writes each array once, in sequence.
//
// A text of long repeats (more than n/32 ranks past 64 symbols, or an LCP
// past 8192) takes Kasai's method instead, whose cost does not depend on the
// LCP values.  Kasai's observation: for text positions i and i+1, the LCP of
// suffix i+1 with its rank predecessor is at least the LCP of suffix i with
// its rank predecessor minus one.  It is applied in the "permuted LCP" form:
//   1. one scatter per rank k writes {ISA, PHI} = {k, SA[k-1]} at position
//      SA[k] (one 8-byte write instead of separate ISA / predecessor lookups);
//   2. text positions are walked in order in chunks (h carried within a
//      chunk), comparing T[i+h..] with T[PHI[i]+h..] 32 symbols at a time on
//      the 2-bit copy, and PLCP[i] and ISA[i] are written in text order;
//   3. LCP[ISA[i]] = PLCP[i] is scattered back to rank order.
// The choice is made on the device and read back once (one stream
// synchronisation per call); texts below 2^20 symbols, whose call is bound by
// launches, take Kasai's passes directly.
#include "lcp_kernels.cuh"
#include "radix.cuh"

LOR_DEFINE_TU_STATUS(lor_status_lcp)

namespace lor {
namespace {

// Inputs of at least this many symbols scatter through bucketing (one radix
// pass on the destination's top bits, then writes that combine in L2).
constexpr int64_t kBucketMin = int64_t(1) << 22;
// Texts of at least this many symbols try the direct LCP route first.
constexpr int64_t kDirectMin = int64_t(1) << 20;

__global__ void k_lcp_scatter_direct(const int32_t *__restrict__ isa, int64_t n,
                                     const int32_t *__restrict__ plcp, int32_t *__restrict__ lcp) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t r = isa[i];
    if (r >= 0 && r < n) lcp[r] = plcp[i];
}

// ISA[SA[k]] = k (small texts; larger ones go through the bucketed scatter).
__global__ void k_isa_direct(const int32_t *__restrict__ sa, int64_t n, int32_t *__restrict__ isa, int *status) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t p = sa[k];
    if (p < 0 || p >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        return;
    }
    isa[p] = int32_t(k);
}

struct LcpLayout {
    size_t ip = 0, plcp = 0, ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t kbuf = 0, vbuf = 0, packed = 0, total = 0;
};
LcpLayout lcp_layout(int64_t n) {
    LcpLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ip = take(sizeof(int2) * size_t(n));
    L.plcp = take(sizeof(int32_t) * size_t(n));
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(n);
    L.lookback = take(L.lookback_bytes);
    L.kbuf = take(sizeof(uint32_t) * size_t(n));
    L.vbuf = take(sizeof(uint64_t) * size_t(n));
    L.packed = take(packed_text_bytes(n));
    L.total = off;
    return L;
}

// ---- 64-bit indices (n up to LOR_MAX_N64): positions are held as uint32
// inside (n < 2^32), ISA is written as int64 and LCP stays int32.

// sa32[k] = SA[k] as uint32; an entry outside [0, n) sets LOR_ERR_BAD_INPUT
// and is replaced by k so that later passes stay in bounds.
__global__ void k_narrow_sa64(const int64_t *__restrict__ sa, int64_t n, uint32_t *__restrict__ sa32, int *status) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = sa[k];
    if (p < 0 || p >= n) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        p = k;
    }
    sa32[k] = uint32_t(p);
}

// The PLCP pass of k_plcp_packed for 64-bit texts: {ISA, PHI} as uint32
// pairs (PHI 0xFFFFFFFF: no predecessor), the bitmap comparison only (the
// exception list holds int32 positions), ISA written as int64 and as uint32
// (the keys of the LCP scatter).  A PLCP value above INT32_MAX sets
// LOR_ERR_TOO_LARGE and is clamped.
__global__ void __launch_bounds__(kPlcpThreads) k_plcp64(const uint8_t *__restrict__ t, PackedText T, int64_t n,
                                                         const uint2 *__restrict__ ip, int64_t *__restrict__ isa,
                                                         uint32_t *__restrict__ isa32, int32_t *__restrict__ plcp,
                                                         int *status) {
    __shared__ uint32_t s_phi[kPlcpTile];
    __shared__ int32_t s_h[kPlcpTile];
    const int64_t base = int64_t(blockIdx.x) * kPlcpTile;
    const int cnt = int(min64(int64_t(kPlcpTile), n - base));
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) {
        const uint2 v = ip[base + i];
        isa[base + i] = int64_t(v.x);
        isa32[base + i] = v.x;
        s_phi[i] = v.y;
    }
    __syncthreads();
    int64_t h = 0;
    bool bad = false, big = false;
    const int l0 = int(threadIdx.x) * kPlcpPer;
    for (int l = l0; l < l0 + kPlcpPer && l < cnt; ++l) {
        const int64_t i = base + l;
        const uint32_t phi = s_phi[l];
        if (phi == 0xFFFFFFFFu || int64_t(phi) >= n) {
            if (phi != 0xFFFFFFFFu) bad = true;
            h = 0;
            s_h[l] = 0;
            continue;
        }
        h = extend_bitmap(t, T, n, i, int64_t(phi), h);
        if (h > INT32_MAX) big = true;
        s_h[l] = int32_t(h > INT32_MAX ? INT32_MAX : h);
        if (h > 0) --h;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
    if (big) atomicCAS(status, 0, LOR_ERR_TOO_LARGE);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) plcp[base + i] = s_h[i];
}

struct Lcp64Layout {
    size_t ip = 0, plcp = 0, ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t kbuf = 0, vbuf = 0, sa32 = 0, packed = 0, total = 0;
};
Lcp64Layout lcp64_layout(int64_t n) {
    Lcp64Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ip = take(sizeof(uint2) * size_t(n));
    L.plcp = take(sizeof(int32_t) * size_t(n));
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(n);
    L.lookback = take(L.lookback_bytes);
    L.kbuf = take(sizeof(uint32_t) * size_t(n));
    L.vbuf = take(sizeof(uint64_t) * size_t(n));
    L.sa32 = take(sizeof(uint32_t) * size_t(n));
    L.packed = take(packed_text_bytes(n));
    L.total = off;
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
    char *ws = (char *)d_ws;
    int2 *ip = (int2 *)(ws + L.ip);
    int32_t *plcp = (int32_t *)(ws + L.plcp);
    uint32_t *kbuf = (uint32_t *)(ws + L.kbuf);
    uint64_t *vbuf = (uint64_t *)(ws + L.vbuf);
    const bool bucket = n >= kBucketMin;
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl);
    rs.max_tiles = cdiv(n, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    const PackedText T = packed_text_at(ws + L.packed, n);
    {
        // text read twice, 2-bit copy and exception bitmap written
        ProfScope ps(PK_KASAI, double(n) * (2 + 0.375), s);
        const int rc = pack_text(d_text, n, T, s);
        if (rc) return rc;
    }
    // Texts below kDirectMin symbols take Kasai's passes at once: there the
    // call is bound by launches and the route's read-back would cost more
    // than it saves.
    int fallback = n < kDirectMin ? 1 : 0;
    if (!fallback) {
        // LCP in rank order by direct comparison (the long list in the PLCP
        // buffer), then the ranks that reached the cap
        LOR_CUDA_TRY(cudaMemsetAsync(T.ctl + kCtlLong, 0, 2 * sizeof(int), s));
        {
            // SA read, LCP written, two 16-symbol windows of the 2-bit copy
            ProfScope ps(PK_KASAI, double(n) * (4 + 4 + 8), s);
            k_lcp_direct<<<unsigned(min64(cdiv(cdiv(n, kLcpPer), kLcpThreads), 152 * 8)), kLcpThreads, 0, s>>>(
                d_text, T, n, d_sa, d_lcp, reinterpret_cast<uint32_t *>(plcp), status);
            LOR_LAUNCH_CHECK();
        }
        const int64_t max_long = n / 32 + 64;
        {
            ProfScope ps(PK_KASAI, 0.0, s);
            k_lcp_long<<<unsigned(min64(cdiv(max_long, 256), 152 * 8)), 256, 0, s>>>(
                d_text, T, n, d_sa, d_lcp, reinterpret_cast<const uint32_t *>(plcp), max_long);
            LOR_LAUNCH_CHECK();
        }
        LOR_CUDA_TRY(cudaMemcpyAsync(&fallback, T.ctl + kCtlFallback, sizeof(int), cudaMemcpyDeviceToHost, s));
        LOR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (bucket) {
        LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
        LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    }
    if (!fallback) {
        // ISA[SA[k]] = k
        if (bucket) {
            uint32_t *vb0 = reinterpret_cast<uint32_t *>(vbuf);
            return bucketed_scatter(rs, (const uint32_t *)d_sa, nullptr, n, n, kbuf, vb0, vb0 + n, d_isa, 0,
                                    PK_ISA_SCATTER);
        }
        ProfScope ps(PK_ISA_SCATTER, double(n) * 8, s);
        k_isa_direct<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, d_isa, status);
        LOR_LAUNCH_CHECK();
        return LOR_OK;
    }
    // A text of long repeats: the permuted Kasai passes (cost independent of
    // the LCP values).
    if (bucket) {
        const int rc = bucketed_isa_phi(rs, d_sa, n, n, kbuf, vbuf, ip);
        if (rc) return rc;
    } else {
        // SA read (4 + 4 neighbour), 8-byte scatter
        ProfScope ps(PK_ISA_SCATTER, double(n) * 12, s);
        k_isa_phi<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, nullptr, ip, status);
        LOR_LAUNCH_CHECK();
    }
    {
        // {ISA, PHI} read, ISA + PLCP written, two text windows per position
        ProfScope ps(PK_KASAI, double(n) * (8 + 4 + 4 + 2), s);
        k_plcp_packed<<<unsigned(cdiv(n, kPlcpTile)), kPlcpThreads, 0, s>>>(d_text, T, n, ip, d_isa, plcp, status);
    }
    LOR_LAUNCH_CHECK();
    // LCP[ISA[i]] = PLCP[i]
    if (bucket) {
        uint32_t *vb0 = reinterpret_cast<uint32_t *>(vbuf);
        const int rc = bucketed_scatter(rs, (const uint32_t *)d_isa, (const uint32_t *)plcp, n, n, kbuf, vb0,
                                        vb0 + n, d_lcp, 0);
        if (rc) return rc;
    } else {
        ProfScope ps(PK_KASAI, double(n) * 12, s);
        k_lcp_scatter_direct<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_isa, n, plcp, d_lcp);
        LOR_LAUNCH_CHECK();
    }
    return LOR_OK;
}

extern "C" size_t lor_lcp64_workspace_size(int64_t n) {
    if (n < 1 || n > LOR_MAX_N64) return 0;
    return lcp64_layout(n).total;
}

extern "C" int lor_lcp64(const uint8_t *d_text, const int64_t *d_sa, int64_t n, int64_t *d_isa, int32_t *d_lcp,
                         void *d_ws, size_t ws_bytes, lor_stream_t stream) {
    if (!d_text || !d_sa || !d_isa || !d_lcp || n < 1) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N64) return LOR_ERR_TOO_LARGE;
    const Lcp64Layout L = lcp64_layout(n);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    char *ws = (char *)d_ws;
    uint2 *ip = (uint2 *)(ws + L.ip);
    int32_t *plcp = (int32_t *)(ws + L.plcp);
    uint32_t *kbuf = (uint32_t *)(ws + L.kbuf);
    uint64_t *vbuf = (uint64_t *)(ws + L.vbuf);
    uint32_t *sa32 = (uint32_t *)(ws + L.sa32);
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl);
    rs.max_tiles = cdiv(n, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    {
        ProfScope ps(PK_ISA_SCATTER, double(n) * (8 + 4), s);
        k_narrow_sa64<<<unsigned(cdiv(n, 256)), 256, 0, s>>>(d_sa, n, sa32, status);
        LOR_LAUNCH_CHECK();
    }
    // {ISA, PHI}[SA[k]] = {k, SA[k-1]} (0xFFFFFFFF for k = 0) through one
    // partition pass on the destination's top bits.
    int rc = bucketed_isa_phi(rs, reinterpret_cast<const int32_t *>(sa32), n, n, kbuf, vbuf,
                              reinterpret_cast<int2 *>(ip));
    if (rc) return rc;
    const PackedText T = packed_text_at(ws + L.packed, n);
    {
        ProfScope ps(PK_KASAI, double(n) * (2 + 0.375), s);
        rc = pack_text(d_text, n, T, s);
        if (rc) return rc;
    }
    {
        // {ISA, PHI} read, ISA (8 + 4) and PLCP written, two text windows per position
        ProfScope ps(PK_KASAI, double(n) * (8 + 12 + 4 + 2), s);
        k_plcp64<<<unsigned(cdiv(n, kPlcpTile)), kPlcpThreads, 0, s>>>(d_text, T, n, ip, d_isa, sa32, plcp, status);
        LOR_LAUNCH_CHECK();
    }
    // LCP[ISA[i]] = PLCP[i]
    uint32_t *vb0 = reinterpret_cast<uint32_t *>(vbuf);
    return bucketed_scatter(rs, sa32, reinterpret_cast<const uint32_t *>(plcp), n, n, kbuf, vb0, vb0 + n, d_lcp, 0);
}
