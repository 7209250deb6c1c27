// sa64.cu -- suffix array of texts beyond the int32 index range (up to
// LOR_MAX_N64 symbols), with 64-bit indices at the boundary.
//
// The suffix order is the one of Section 3 (Tables 1-3); the method here is
// prefix doubling -- the finisher this library's DC3 applies to its reduced
// strings -- started directly on the text:
//   round 0: every suffix gets the key of its first K symbols (K * bits <= 64,
//            bits per code), one LSD radix sort (Section 4, Algorithm 1)
//            orders all n suffixes by it;
//   settle:  a group of equal keys occupies SA indices [g, g + size); every
//            member's rank becomes g (the number of suffixes with a smaller
//            prefix), a group of one is final (SA[g] = its position);
//   round r: the members of unresolved groups, kept in SA order, are sorted
//            by (their group, rank[pos + h]) with h = K * 2^(r-1) -- the rank
//            of the suffix h symbols on, so the order by the first 2h symbols
//            -- and settled again, until no group is left.
// Inside the library every position is held as uint32 (n < 2^32): the sort
// passes move 4-byte values instead of 8; SA is written as int64.
#include "radix.cuh"
#include "scan.cuh"

LOR_DEFINE_TU_STATUS(lor_status_sa64)

namespace lor {
namespace {

constexpr int kK0Threads = 256;
constexpr int kK0Per = 8;  // consecutive positions per thread
constexpr int kK0Tile = kK0Threads * kK0Per;
constexpr int kK0Halo = 64;  // K <= 64 symbols of look-ahead

// keys[i] = the first K codes of suffix i, `bits` bits each, most
// significant first, 0 past the end of the text (0 sorts below every code).
// A code outside [1, sigma) sets LOR_ERR_BAD_SYMBOL and is clamped into range
// so that it cannot spill into the neighbouring fields of the key.
__global__ void __launch_bounds__(kK0Threads) k_sa64_keys0(const uint8_t *__restrict__ t, int64_t n, int sigma,
                                                           int bits, int K, uint64_t *__restrict__ keys,
                                                           int *status) {
    __shared__ uint8_t st[kK0Tile + kK0Halo];
    const int64_t base = int64_t(blockIdx.x) * kK0Tile;
    bool bad = false;
    for (int l = threadIdx.x; l < kK0Tile + kK0Halo; l += kK0Threads) {
        const int64_t i = base + l;
        int c = 0;
        if (i < n) {
            c = t[i];
            if (c < 1 || c >= sigma) {
                bad = true;
                c = c < 1 ? 1 : sigma - 1;
            }
        }
        st[l] = uint8_t(c);
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
    __syncthreads();
    const int l0 = int(threadIdx.x) * kK0Per;
    const uint64_t mask = K * bits >= 64 ? ~uint64_t(0) : (uint64_t(1) << (K * bits)) - 1;
    uint64_t key = 0;
    for (int j = 0; j < K; ++j) key = (key << bits) | st[l0 + j];
    uint64_t out[kK0Per];
#pragma unroll
    for (int u = 0; u < kK0Per; ++u) {
        out[u] = key;
        key = ((key << bits) | st[l0 + u + K]) & mask;
    }
    const int64_t i0 = base + l0;
    if (i0 + kK0Per <= n) {
        ulonglong2 *q = reinterpret_cast<ulonglong2 *>(keys + i0);  // i0 is a multiple of 8
#pragma unroll
        for (int u = 0; u < kK0Per / 2; ++u) q[u] = make_ulonglong2(out[2 * u], out[2 * u + 1]);
    } else {
        for (int u = 0; u < kK0Per; ++u)
            if (i0 + u < n) keys[i0 + u] = out[u];
    }
}

// Group names over the sorted keys: name[j] = number of group heads at or
// before j; H[name - 1] = the index of that head.
__global__ void __launch_bounds__(kScanThreads) k_sa64_names(const uint64_t *__restrict__ ks, int64_t m,
                                                             uint32_t *__restrict__ name, uint32_t *__restrict__ H,
                                                             uint32_t *n_names, uint64_t *lb,
                                                             unsigned long long *ctr, unsigned long long tile_base,
                                                             uint32_t epoch, int *status) {
    auto is_head = [&](int64_t j) { return j == 0 || ks[j] != ks[j - 1]; };
    tile_names(
        m, is_head,
        [&](int64_t j, uint32_t nm) {
            name[j] = nm;
            if (is_head(j)) H[nm - 1] = uint32_t(j);
        },
        n_names, lb, ctr, tile_base, epoch, status);
}

// Settle and compact in one pass over the m sorted items.  Item j (position
// vs[j], SA index gk[j], or j itself in round 0) takes the rank of its group,
// the SA index of the group's head; a group of one writes its final SA entry.
// Members of larger groups are appended, in order, to the next round's list:
// position, SA index, and (in ukey) the list index of their group's first
// member, from which the next sort key is made.
__global__ void __launch_bounds__(kScanThreads) k_sa64_settle(
    const uint32_t *__restrict__ name, const uint32_t *__restrict__ H, int64_t m, const uint32_t *__restrict__ vs,
    const uint32_t *__restrict__ gk, uint32_t *__restrict__ rank, int64_t *__restrict__ sa,
    uint64_t *__restrict__ ukey, uint32_t *__restrict__ upos, uint32_t *__restrict__ ugk, uint32_t *count,
    uint64_t *lb, unsigned long long *ctr, unsigned long long tile_base, uint32_t epoch, int *status,
    int64_t ntiles) {
    tile_compact(
        m,
        [&](int64_t j) {
            const uint32_t nm = name[j];
            const uint32_t jh = H[nm - 1];
            const bool single = int64_t(jh) == j && (j + 1 == m || name[j + 1] != nm);
            const uint32_t g = gk ? gk[jh] : jh;
            const uint32_t p = vs[j];
            rank[p] = g;
            if (single) sa[gk ? gk[j] : uint32_t(j)] = int64_t(p);
            return !single;
        },
        [&](int64_t j, uint32_t o) {
            const uint32_t jh = H[name[j] - 1];
            ukey[o] = uint64_t(o) - uint64_t(j - int64_t(jh));
            upos[o] = vs[j];
            ugk[o] = gk ? gk[j] : uint32_t(j);
        },
        lb, ctr, tile_base, epoch, status, count, ntiles);
}

// Next sort key of list item o: (group's first list index) << lo_bits |
// (rank of the suffix h symbols on, plus one; 0 past the end of the text).
__global__ void k_sa64_round_keys(uint64_t *__restrict__ ukey, const uint32_t *__restrict__ upos, int64_t U,
                                  const uint32_t *__restrict__ rank, int64_t n, int64_t h, int lo_bits) {
    const int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (o >= U) return;
    const int64_t q = int64_t(upos[o]) + h;
    const uint64_t k2 = q < n ? uint64_t(rank[q]) + 1 : 0;
    ukey[o] = (ukey[o] << lo_bits) | k2;
}

struct Sa64Layout {
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0;
    size_t k0 = 0, k1 = 0, v0 = 0, v1 = 0, name = 0, H = 0, rank = 0, g0 = 0, g1 = 0, total = 0;
};

Sa64Layout sa64_layout(int64_t n) {
    Sa64Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t N = size_t(n);
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(n);
    L.lookback = take(L.lookback_bytes);
    L.k0 = take(sizeof(uint64_t) * N);
    L.k1 = take(sizeof(uint64_t) * N);
    L.v0 = take(sizeof(uint32_t) * N);
    L.v1 = take(sizeof(uint32_t) * N);
    L.name = take(sizeof(uint32_t) * N);
    L.H = take(sizeof(uint32_t) * N);
    L.rank = take(sizeof(uint32_t) * N);
    L.g0 = take(sizeof(uint32_t) * N);
    L.g1 = take(sizeof(uint32_t) * N);
    L.total = off;
    return L;
}

// Names then settle over m sorted items; returns the size of the next list.
int sa64_settle_round(RadixScratch &rs, const uint64_t *ks, const uint32_t *vs, const uint32_t *gk, int64_t m,
                      uint32_t *name, uint32_t *H, uint32_t *rank, int64_t *sa, uint64_t *ukey, uint32_t *upos,
                      uint32_t *ugk, uint32_t *ctl, int64_t *U_out) {
    cudaStream_t s = rs.stream;
    const int64_t ntiles = cdiv(m, kScanTile);
    {
        ProfScope ps(PK_NAMING, double(m) * (8 + 4 + 4), s);
        rs.epoch++;
        k_sa64_names<<<unsigned(ntiles), kScanThreads, 0, s>>>(ks, m, name, H, ctl, rs.lookback, rs.tile_ctr,
                                                               rs.tile_base, rs.epoch, rs.status);
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
    }
    {
        // name, head, position read; rank scattered, SA written
        ProfScope ps(PK_RANK_SCATTER, double(m) * (4 + 4 + 4 + 4 + 8), s);
        rs.epoch++;
        k_sa64_settle<<<unsigned(ntiles), kScanThreads, 0, s>>>(name, H, m, vs, gk, rank, sa, ukey, upos, ugk,
                                                                ctl + 1, rs.lookback, rs.tile_ctr, rs.tile_base,
                                                                rs.epoch, rs.status, ntiles);
        LOR_LAUNCH_CHECK();
        rs.tile_base += (unsigned long long)ntiles;
    }
    uint32_t h_u = 0;
    LOR_CUDA_TRY(cudaMemcpyAsync(&h_u, ctl + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaStreamSynchronize(s));
    *U_out = int64_t(h_u);
    return LOR_OK;
}

}  // namespace
}  // namespace lor

using namespace lor;

extern "C" size_t lor_build_sa64_workspace_size(int64_t n, int32_t sigma) {
    if (n < 1 || n > LOR_MAX_N64 || sigma < 2 || sigma > 256) return 0;
    return sa64_layout(n).total;
}

extern "C" int lor_build_sa64(const uint8_t *d_text, int64_t n, int32_t sigma, int64_t *d_sa, void *d_ws,
                              size_t ws_bytes, lor_stream_t stream) {
    if (!d_text || !d_sa || n < 1 || sigma < 2 || sigma > 256) return LOR_ERR_INVALID_ARG;
    if (n > LOR_MAX_N64) return LOR_ERR_TOO_LARGE;
    const Sa64Layout L = sa64_layout(n);
    if (!d_ws || ws_bytes < L.total || (uintptr_t(d_ws) & 255)) return LOR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    char *ws = (char *)d_ws;
    RadixScratch rs;
    rs.hist = (uint32_t *)(ws + L.hist);
    rs.offsets = (uint32_t *)(ws + L.offsets);
    rs.lookback = (uint64_t *)(ws + L.lookback);
    rs.tile_ctr = (unsigned long long *)(ws + L.ctrl);
    rs.max_tiles = cdiv(n, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    uint32_t *ctl = (uint32_t *)(ws + L.ctrl + 128);
    uint64_t *k0 = (uint64_t *)(ws + L.k0), *k1 = (uint64_t *)(ws + L.k1);
    uint32_t *v0 = (uint32_t *)(ws + L.v0), *v1 = (uint32_t *)(ws + L.v1);
    uint32_t *name = (uint32_t *)(ws + L.name), *H = (uint32_t *)(ws + L.H), *rank = (uint32_t *)(ws + L.rank);
    uint32_t *gA = (uint32_t *)(ws + L.g0), *gB = (uint32_t *)(ws + L.g1);
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));

    const int bits = bit_width_u64(uint64_t(sigma - 1));
    const int K = 64 / bits;
    {
        ProfScope ps(PK_SAMPLE_KEYS, double(n) * (1 + 8), s);
        k_sa64_keys0<<<unsigned(cdiv(n, kK0Tile)), kK0Threads, 0, s>>>(d_text, n, sigma, bits, K, k0, status);
        LOR_LAUNCH_CHECK();
    }
    uint64_t *ks;
    uint32_t *vs;
    int rc = radix_sort_pairs<uint64_t>(rs, k0, v0, k1, v1, n, 0, K * bits, true, &ks, &vs);
    if (rc) return rc;
    // The next list goes to whichever key/value buffers the sort left free.
    uint64_t *uk = ks == k0 ? k1 : k0;
    uint32_t *up = vs == v0 ? v1 : v0;
    int64_t U = 0;
    rc = sa64_settle_round(rs, ks, vs, nullptr, n, name, H, rank, d_sa, uk, up, gA, ctl, &U);
    if (rc) return rc;
    const int lo_bits = bit_width_u64(uint64_t(n));  // rank + 1 <= n
    int64_t h = K, m = n;
    uint32_t *g_in = gA, *g_out = gB;
    for (int round = 1; U > 0; ++round) {
        // Every unresolved group has two or more members; a list longer than
        // the previous one, or rounds past the doubling bound, mean that a
        // bounded wait gave up (the status word says which).
        if (U > m || U < 2 || h > 2 * n + 64 || round > 40) return LOR_ERR_TIMEOUT;
        {
            ProfScope ps(PK_SAMPLE_KEYS, double(U) * (8 + 4 + 4 + 8), s);
            k_sa64_round_keys<<<unsigned(cdiv(U, 256)), 256, 0, s>>>(uk, up, U, rank, n, h, lo_bits);
            LOR_LAUNCH_CHECK();
        }
        uint64_t *kspare = uk == k0 ? k1 : k0;
        uint32_t *vspare = up == v0 ? v1 : v0;
        const int end_bit = lo_bits + bit_width_u64(uint64_t(U - 1));
        rc = radix_sort_pairs<uint64_t>(rs, uk, up, kspare, vspare, U, 0, end_bit, false, &ks, &vs);
        if (rc) return rc;
        uk = ks == k0 ? k1 : k0;
        up = vs == v0 ? v1 : v0;
        m = U;
        rc = sa64_settle_round(rs, ks, vs, g_in, m, name, H, rank, d_sa, uk, up, g_out, ctl, &U);
        if (rc) return rc;
        uint32_t *t = g_in;
        g_in = g_out;
        g_out = t;
        h *= 2;
    }
    return LOR_OK;
}
