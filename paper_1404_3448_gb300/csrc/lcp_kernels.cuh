// lcp_kernels.cuh -- the LCP kernels (Section 3, LCP table; Kasai et
// al., cited there), shared by lor_lcp and the batched pipeline:
//   k_isa_phi   {ISA, PHI} = {k, SA[k-1]} scattered to position SA[k];
//   k_text_max, k_pack_text: a 2-bit copy of the text (the four largest
//               codes; smaller codes such as terminators are flagged in an
//               exception bitmap and compared as bytes).  For DNA the copy is
//               a quarter of the text and stays in L2, where the random
//               PHI-side reads of the next kernel land;
//   k_plcp_packed text positions in order (h carried within a chunk),
//               comparing T[i+h..] with T[PHI[i]+h..] 32 symbols at a time:
//               ISA and PLCP in text order;
//   k_lcp_gather LCP[k] = PLCP[SA[k]].
#pragma once

#include <climits>

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

constexpr int kPlcpThreads = 256;
constexpr int kPlcpPer = 16;  // text positions per thread
constexpr int kPlcpTile = kPlcpThreads * kPlcpPer;

// ---- packed text

constexpr int kPackThreads = 256;
constexpr int kPackPer = 32;  // symbols per thread: one 64-bit word, one 32-bit exception word
constexpr int kPackTile = kPackThreads * kPackPer;
constexpr int kExcCap = 4096;    // exceptions kept as a sorted list (else the bitmap is used)
constexpr int kExcShared = 512;  // listed exceptions the LCP kernel keeps in shared memory

// Words of the 2-bit copy and of the exception bitmap for n symbols (enough
// for 16-byte loads of the chunk holding any symbol, and for two-word
// windows at any position).
__host__ __device__ inline int64_t packed_words(int64_t n) { return n / 32 + 4; }

// The 2-bit copy of a text: P (16-byte aligned), the exception bitmap E,
// the sorted exception list (when it has at most kExcCap entries), and two
// control words: ctl[0] = largest code, ctl[1] = number of exceptions.
struct PackedText {
    uint64_t *P;
    uint32_t *E;
    int32_t *list;
    int *ctl;
};

inline size_t packed_text_bytes(int64_t n) {
    return align256(sizeof(uint64_t) * size_t(packed_words(n))) +
           align256(sizeof(uint32_t) * size_t(packed_words(n))) + align256(sizeof(int32_t) * kExcCap) + 256;
}
inline PackedText packed_text_at(char *mem, int64_t n) {
    PackedText T;
    size_t off = 0;
    T.P = (uint64_t *)(mem + off);
    off += align256(sizeof(uint64_t) * size_t(packed_words(n)));
    T.E = (uint32_t *)(mem + off);
    off += align256(sizeof(uint32_t) * size_t(packed_words(n)));
    T.list = (int32_t *)(mem + off);
    off += align256(sizeof(int32_t) * kExcCap);
    T.ctl = (int *)(mem + off);
    return T;
}

// ctl[0] = largest code in the text (the caller zeroes it first).
__global__ void k_text_max(const uint8_t *__restrict__ t, int64_t n, int *mx) {
    uint32_t m = 0;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    int64_t head = 0;
    if ((uintptr_t(t) & 15) == 0) {
        // 16 bytes per load; per-byte maximum of four packed bytes via __vmaxu4
        const int64_t nv = n / 16;
        const uint4 *v = reinterpret_cast<const uint4 *>(t);
        uint32_t acc = 0;
        for (int64_t i = tid; i < nv; i += nth) {
            const uint4 x = v[i];
            acc = __vmaxu4(acc, __vmaxu4(__vmaxu4(x.x, x.y), __vmaxu4(x.z, x.w)));
        }
        m = max(max(acc & 0xFFu, (acc >> 8) & 0xFFu), max((acc >> 16) & 0xFFu, acc >> 24));
        head = nv * 16;
    }
    for (int64_t i = head + tid; i < n; i += nth) m = max(m, uint32_t(t[i]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, int(m));
}

// Code c in [mx-3, mx] -> c - (mx - 3) in two bits (symbol k of a word in
// bits 2k, 2k+1); any smaller code -> 0 with its exception bit set and its
// position appended to the (unordered) exception list.
__global__ void __launch_bounds__(kPackThreads) k_pack_text(const uint8_t *__restrict__ t, int64_t n,
                                                            PackedText T) {
    __shared__ uint8_t st[kPackTile];
    const int64_t base = int64_t(blockIdx.x) * kPackTile;
    const int cnt = int(min64(int64_t(kPackTile), n - base));
    for (int i = threadIdx.x; i < cnt; i += kPackThreads) st[i] = t[base + i];
    __syncthreads();
    const int lo = T.ctl[0] - 3;
    uint64_t w = 0;
    uint32_t e = 0;
    const int l0 = int(threadIdx.x) * kPackPer;
#pragma unroll 8
    for (int k = 0; k < kPackPer; ++k) {
        const int l = l0 + k;
        if (l >= cnt) break;
        const int c = int(st[l]) - lo;
        if (c >= 0) w |= uint64_t(c & 3) << (2 * k);
        else e |= 1u << k;
    }
    const int64_t wi = int64_t(blockIdx.x) * kPackThreads + threadIdx.x;
    if (l0 < cnt) {
        T.P[wi] = w;
        T.E[wi] = e;
    }
    if (e) {
        int slot = atomicAdd(&T.ctl[1], __popc(e));
        for (; e && slot < kExcCap; e &= e - 1, ++slot) T.list[slot] = int32_t(base + l0 + __ffs(int(e)) - 1);
    }
}

// Sorts the exception list in place when it is short enough to be used.
__global__ void __launch_bounds__(1024) k_sort_exc(PackedText T) {
    __shared__ int32_t v[kExcCap];
    const int cnt = T.ctl[1];
    if (cnt <= 1 || cnt > kExcCap) return;
    int m = 1;
    while (m < cnt) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = i < cnt ? T.list[i] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    if ((v[i] > v[l]) == up) {
                        const int32_t x = v[i];
                        v[i] = v[l];
                        v[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) T.list[i] = v[i];
}

// Enqueues the 2-bit copy of t[0..n) (the buffers of T come from
// packed_text_at) on stream s.
inline int pack_text(const uint8_t *t, int64_t n, const PackedText &T, cudaStream_t s) {
    const int64_t w0 = n / 32;
    LOR_CUDA_TRY(cudaMemsetAsync(T.P + w0, 0, sizeof(uint64_t) * size_t(packed_words(n) - w0), s));
    LOR_CUDA_TRY(cudaMemsetAsync(T.E + w0, 0, sizeof(uint32_t) * size_t(packed_words(n) - w0), s));
    LOR_CUDA_TRY(cudaMemsetAsync(T.ctl, 0, 2 * sizeof(int), s));
    k_text_max<<<unsigned(min64(cdiv(n, 256), 152 * 8)), 256, 0, s>>>(t, n, T.ctl);
    LOR_LAUNCH_CHECK();
    k_pack_text<<<unsigned(cdiv(n, kPackTile)), kPackThreads, 0, s>>>(t, n, T);
    LOR_LAUNCH_CHECK();
    k_sort_exc<<<1, 1024, 0, s>>>(T);
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

// Symbols p .. p+31 of the 2-bit copy (p + 32 <= n) and their exception bits.
__device__ __forceinline__ uint64_t window2(const uint64_t *__restrict__ P, int64_t p) {
    const int64_t w = p >> 5;
    const int sft = int(p & 31) * 2;
    const uint64_t a = P[w];
    return sft ? (a >> sft) | (P[w + 1] << (64 - sft)) : a;
}
__device__ __forceinline__ uint32_t window_exc(const uint32_t *__restrict__ E, int64_t p) {
    const int64_t w = p >> 5;
    return __funnelshift_r(E[w], E[w + 1], uint32_t(p & 31));
}

// Symbols from p on out of the 16-byte chunk holding p: 32 of them when p
// sits in the chunk's first half, else the 64 - (p mod 64) up to its end.
__device__ __forceinline__ uint64_t window_chunk(const uint64_t *__restrict__ P, int64_t p, int &avail,
                                                 uint64_t keep) {
    const ulonglong2 v = ld_u64x2_hint(reinterpret_cast<const ulonglong2 *>(P) + (p >> 6), keep);
    const int off = int(p & 63);
    if (off < 32) {
        avail = 32;
        return off ? (v.x >> (2 * off)) | (v.y << (64 - 2 * off)) : v.x;
    }
    avail = 64 - off;
    return v.y >> (2 * (off - 32));
}

// First exception at or after p (n if none), from the sorted list.
__device__ __forceinline__ int64_t next_exc(const int32_t *__restrict__ lst, int cnt, int64_t p, int64_t n) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lst[mid] < p) lo = mid + 1;
        else hi = mid;
    }
    return lo < cnt ? int64_t(lst[lo]) : n;
}

// 32-bit forms of window_chunk and next_exc for texts below 2^31 symbols
// (the int32 path): position arithmetic in 32 bits halves the ALU work of
// the comparison loop, which bounds the PLCP pass.
__device__ __forceinline__ uint64_t window_chunk32(const uint64_t *__restrict__ P, uint32_t p, int &avail,
                                                   uint64_t keep) {
    const ulonglong2 v = ld_u64x2_hint(reinterpret_cast<const ulonglong2 *>(P) + (p >> 6), keep);
    const uint32_t off = p & 63u;
    if (off < 32) {
        avail = 32;
        return off ? (v.x >> (2 * off)) | (v.y << (64 - 2 * off)) : v.x;
    }
    avail = int(64 - off);
    return v.y >> (2 * (off - 32));
}

__device__ __forceinline__ int32_t next_exc32(const int32_t *__restrict__ lst, int cnt, int32_t p, int32_t n) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lst[mid] < p) lo = mid + 1;
        else hi = mid;
    }
    return lo < cnt ? lst[lo] : n;
}

// lcp(T[i..], T[j..]) given that the first h symbols match: 32 symbols at a
// time on the 2-bit copy, with the exception bitmap marking the symbols that
// must be compared as bytes.
__device__ __forceinline__ int64_t extend_bitmap(const uint8_t *__restrict__ t, const PackedText &T, int64_t n,
                                                 int64_t i, int64_t j, int64_t h) {
    while (i + h + 32 <= n && j + h + 32 <= n) {
        const uint64_t d = window2(T.P, i + h) ^ window2(T.P, j + h);
        const uint32_t e = window_exc(T.E, i + h) | window_exc(T.E, j + h);
        const int dpos = d ? (__ffsll((long long)d) - 1) >> 1 : 32;
        const int epos = e ? __ffs(int(e)) - 1 : 32;
        if (dpos < epos) return h + dpos;
        if (epos < 32) {
            h += epos;
            if (t[i + h] != t[j + h]) return h;
            ++h;
        } else {
            h += 32;
        }
    }
    while (i + h < n && j + h < n && t[i + h] == t[j + h]) ++h;
    return h;
}

// Shared-memory index of position l of a tile: one pad word per 16, so that
// the 16-position chunks of a warp's threads fall in different banks.
__device__ __forceinline__ int chunk_slot(int l) { return l + (l >> 4); }

__global__ void __launch_bounds__(kPlcpThreads) k_plcp_packed(const uint8_t *__restrict__ t, PackedText T,
                                                              int64_t n, const int2 *__restrict__ ip,
                                                              int32_t *__restrict__ isa,
                                                              int32_t *__restrict__ plcp, int *status) {
    __shared__ int32_t s_out[kPlcpTile + kPlcpTile / 16];
    __shared__ int32_t s_exc[kExcShared];
    const int64_t base = int64_t(blockIdx.x) * kPlcpTile;
    const int cnt = int(min64(int64_t(kPlcpTile), n - base));
    const int nexc = T.ctl[1];
    const bool listed = nexc <= kExcCap;
    const int32_t *lst = nexc <= kExcShared ? s_exc : T.list;
    if (nexc <= kExcShared)
        for (int i = threadIdx.x; i < nexc; i += kPlcpThreads) s_exc[i] = T.list[i];
    // The packed text is read at random positions (the PHI side) and should
    // stay in L2; the {ISA, PHI} pairs, ISA and PLCP stream through once.
    const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
    // ISA in text order (coalesced), PHI staged beside the output slots.
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) {
        const int2 v = ld_i32x2_hint(ip + base + i, once);
        st_i32_hint(isa + base + i, v.x, once);
        s_out[chunk_slot(i)] = v.y;
    }
    __syncthreads();
    const uint64_t *__restrict__ P = T.P;
    int64_t h = 0;
    bool bad = false;
    const int l0 = int(threadIdx.x) * kPlcpPer;
    int32_t ea = -1;  // first exception at or after the text-order side (valid while a <= ea)
    for (int l = l0; l < l0 + kPlcpPer && l < cnt; ++l) {
        const int64_t i = base + l;
        const int64_t j = s_out[chunk_slot(l)];
        if (j < 0 || j >= n) {
            if (j != -1) bad = true;
            h = 0;
            s_out[chunk_slot(l)] = 0;
            continue;
        }
        if (listed) {
            // Compare packed symbols up to the next exception (or the end) on
            // either side; there compare the bytes and go on if they match.
            // (32-bit positions: n < 2^31 on this path.)  The next exception
            // on the text-order side only moves forward, so it is kept.
            const int32_t n32 = int32_t(n), i32 = int32_t(i), j32 = int32_t(j);
            int32_t h32 = int32_t(h);
            for (;;) {
                const int32_t a = i32 + h32, b = j32 + h32;
                if (a > ea) ea = next_exc32(lst, nexc, a, n32);
                const int32_t lim = min(min(ea - a, next_exc32(lst, nexc, b, n32) - b), min(n32 - a, n32 - b));
                int32_t k = 0;
                bool mism = false;
                while (k < lim) {
                    int aa, ab;
                    const uint64_t wa = window_chunk32(P, uint32_t(a + k), aa, keep);
                    const uint64_t wb = window_chunk32(P, uint32_t(b + k), ab, keep);
                    int len = aa < ab ? aa : ab;
                    if (lim - k < len) len = lim - k;
                    uint64_t d = wa ^ wb;
                    if (len < 32) d &= (uint64_t(1) << (2 * len)) - 1;
                    if (d) {
                        k += (__ffsll((long long)d) - 1) >> 1;
                        mism = true;
                        break;
                    }
                    k += len;
                }
                h32 += k;
                if (mism || i32 + h32 >= n32 || j32 + h32 >= n32 || t[i32 + h32] != t[j32 + h32]) break;
                ++h32;
            }
            h = h32;
        } else {
            h = extend_bitmap(t, T, n, i, j, h);
        }
        s_out[chunk_slot(l)] = int32_t(h);
        if (h > 0) --h;
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kPlcpThreads) st_i32_hint(plcp + base + i, s_out[chunk_slot(i)], once);
}

// ---- LCP in rank order by direct comparison
//
// On text without long repeats the LCP of two suffixes adjacent in the
// suffix array is short (about log4 n symbols for uniform DNA), so comparing
// them directly on the 2-bit copy -- which stays in L2 -- finds almost every
// LCP[k] in one or two 16-byte reads per side, with no scatter to text order
// and back.  k_lcp_direct compares up to kLcpCap symbols; the ranks that
// reach the cap are listed and k_lcp_long goes on to kLcpBudget symbols.
// When the list or a comparison outgrows those bounds (a text of long
// repeats) the caller runs the permuted Kasai passes instead, whose cost does
// not depend on the LCP values.
constexpr int kLcpCap = 64;
constexpr int kLcpBudget = 8192;
constexpr int kLcpPer = 8;  // ranks per thread of k_lcp_direct
constexpr int kLcpThreads = 256;
// control words of PackedText::ctl used here: the long list's length and the
// fallback flag
constexpr int kCtlLong = 2, kCtlFallback = 3;

// lcp(T[i..], T[j..]) given that the first h symbols match, compared up to
// `cap` symbols (a result of cap means "at least cap").  Symbols are
// compared 32 at a time on the 2-bit copy up to the next listed exception on
// either side, where the bytes are compared (the listed form: at most
// kExcCap exceptions).
__device__ __forceinline__ int32_t lcp_listed(const uint8_t *__restrict__ t, const uint64_t *__restrict__ P,
                                              const int32_t *__restrict__ lst, int nexc, int32_t n, int32_t i,
                                              int32_t j, int32_t h, int32_t cap, uint64_t keep) {
    for (;;) {
        const int32_t a = i + h, b = j + h;
        const int32_t lim = min(min(next_exc32(lst, nexc, a, n) - a, next_exc32(lst, nexc, b, n) - b),
                                min(min(n - a, n - b), cap - h));
        int32_t k = 0;
        while (k < lim) {
            int aa, ab;
            const uint64_t wa = window_chunk32(P, uint32_t(a + k), aa, keep);
            const uint64_t wb = window_chunk32(P, uint32_t(b + k), ab, keep);
            int len = aa < ab ? aa : ab;
            if (lim - k < len) len = lim - k;
            uint64_t d = wa ^ wb;
            if (len < 32) d &= (uint64_t(1) << (2 * len)) - 1;
            if (d) return h + k + ((__ffsll((long long)d) - 1) >> 1);
            k += len;
        }
        h += k;
        if (h >= cap || i + h >= n || j + h >= n || t[i + h] != t[j + h]) return h;
        ++h;  // equal exception codes
    }
}

// The same on the exception bitmap (more than kExcCap exceptions).
__device__ __forceinline__ int32_t lcp_bitmap(const uint8_t *__restrict__ t, const PackedText &T, int32_t n,
                                              int32_t i, int32_t j, int32_t h, int32_t cap) {
    while (h < cap && i + h + 32 <= n && j + h + 32 <= n) {
        const uint64_t d = window2(T.P, i + h) ^ window2(T.P, j + h);
        const uint32_t e = window_exc(T.E, i + h) | window_exc(T.E, j + h);
        const int dpos = d ? (__ffsll((long long)d) - 1) >> 1 : 32;
        const int epos = e ? __ffs(int(e)) - 1 : 32;
        if (dpos < epos) return min(h + dpos, cap);
        if (epos < 32) {
            h += epos;
            if (t[i + h] != t[j + h]) return min(h, cap);
            ++h;
        } else {
            h += 32;
        }
    }
    while (h < cap && i + h < n && j + h < n && t[i + h] == t[j + h]) ++h;
    return min(h, cap);
}

// Symbols p .. p+31 of the 2-bit copy (one 16-byte read, or two when p lies
// in the second half of its chunk).
__device__ __forceinline__ uint64_t window32(const uint64_t *__restrict__ P, uint32_t p, uint64_t keep) {
    const ulonglong2 v = ld_u64x2_hint(reinterpret_cast<const ulonglong2 *>(P) + (p >> 6), keep);
    const uint32_t off = p & 63u;
    if (off < 32) return off ? (v.x >> (2 * off)) | (v.y << (64 - 2 * off)) : v.x;
    if (off == 32) return v.y;
    const ulonglong2 u = ld_u64x2_hint(reinterpret_cast<const ulonglong2 *>(P) + (p >> 6) + 1, keep);
    return (v.y >> (2 * (off - 32))) | (u.x << (64 - 2 * (off - 32)));
}

__device__ __forceinline__ int32_t ld_i32_stream(const int32_t *p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// First listed exception at or after p: the bucket table gives it directly
// unless an exception lies in p's bucket before p (then the list is
// searched).  ne[b] = first exception at or after b << sh.
__device__ __forceinline__ int32_t next_exc_tab(const int32_t *__restrict__ ne, int sh, const int32_t *__restrict__ lst,
                                                int nexc, int32_t p, int32_t n) {
    const int32_t e = ne[p >> sh];
    return e >= p ? e : next_exc32(lst, nexc, p, n);
}

constexpr int kLcpBuckets = 256;

// LCP[k] up to kLcpCap over tiles of kLcpPer * kLcpThreads consecutive
// ranks; a resident grid walks the tiles.  Each warp takes kLcpPer * 32
// consecutive ranks of its tile, 32 at a time (coalesced loads and stores).
// Ranks that reach the cap are appended to `longl` (their LCP is finished by
// k_lcp_long).  LCP[0] = 0.  The 32 symbols at SA[k] are read once, by the
// lane of rank k, and passed to the lane of rank k + 1, whose predecessor
// they are (lane 31's go to lane 0 of the warp's next 32 ranks); a
// comparison that needs more (an exception within 32 symbols, or 32 equal
// symbols) goes on with lcp_listed.  An SA entry outside [0, n) sets
// LOR_ERR_BAD_INPUT and gives LCP 0 at the ranks that read it.
__global__ void __launch_bounds__(kLcpThreads) k_lcp_direct(const uint8_t *__restrict__ t, PackedText T, int64_t n,
                                                            const int32_t *__restrict__ sa, int32_t *__restrict__ lcp,
                                                            uint32_t *__restrict__ longl, int *status) {
    __shared__ int32_t s_exc[kExcShared];
    __shared__ int32_t s_ne[kLcpBuckets];
    const int nexc = T.ctl[1];
    const bool listed = nexc <= kExcCap;
    const int32_t *lst = nexc <= kExcShared ? s_exc : T.list;
    if (nexc <= kExcShared)
        for (int i = threadIdx.x; i < nexc; i += kLcpThreads) s_exc[i] = T.list[i];
    const int32_t n32 = int32_t(n);
    int sh = 0;
    while ((int64_t(kLcpBuckets) << sh) < n) ++sh;
    __syncthreads();
    if (listed)
        for (int b = threadIdx.x; b < kLcpBuckets; b += kLcpThreads) {
            const int64_t p = int64_t(b) << sh;
            s_ne[b] = p < n ? next_exc32(lst, nexc, int32_t(p), n32) : n32;
        }
    __syncthreads();
    const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kTile = kLcpThreads * kLcpPer;
    const int32_t ntiles = int32_t(cdiv(n, kTile));
    bool bad = false;
    for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // this warp's ranks, in 32 bits (n < 2^31)
        const int64_t wb64 = int64_t(tile) * kTile + warp * (32 * kLcpPer);
        if (wb64 >= n) continue;  // warp-uniform
        const int32_t wb = int32_t(wb64);
        // the window of the rank before the warp's first
        int32_t jprev = -1;
        uint64_t wprev = 0;
        if (lane == 0 && wb > 0) {
            jprev = sa[wb - 1];
            if (jprev >= 0 && jprev < n32) wprev = window32(T.P, uint32_t(jprev), keep);
        }
        for (int q = 0; q < kLcpPer; ++q) {
            const int32_t base = wb + q * 32;
            if (base >= n32) break;  // warp-uniform
            const int32_t k = base + lane;
            const bool in = k < n32;
            const int32_t i = in ? ld_i32_stream(sa + k, once) : -1;
            const bool i_ok = i >= 0 && i < n32;
            const uint64_t wi = (in && i_ok) ? window32(T.P, uint32_t(i), keep) : 0;
            // the predecessor's window: from the lane before, or for lane 0
            // the last lane's of the previous 32 ranks
            uint64_t wj = __shfl_up_sync(0xffffffffu, wi, 1);
            int32_t j = __shfl_up_sync(0xffffffffu, i, 1);
            const uint64_t w31 = __shfl_sync(0xffffffffu, wi, 31);
            const int32_t i31 = __shfl_sync(0xffffffffu, i, 31);
            if (lane == 0) {
                wj = wprev;
                j = jprev;
                wprev = w31;
                jprev = i31;
            }
            if (!in) continue;
            int32_t h = 0;
            if (k > 0) {
                if (!i_ok || j < 0 || j >= n32) {
                    bad = true;
                } else {
                    // the windows decide when they differ before an exception on
                    // either side (the bitmap form checks its exceptions itself)
                    uint64_t d = 0;
                    int32_t lim = 0;
                    if (listed) {
                        lim = min(min(min(n32 - i, n32 - j), 32),
                                  min(next_exc_tab(s_ne, sh, lst, nexc, i, n32) - i,
                                      next_exc_tab(s_ne, sh, lst, nexc, j, n32) - j));
                        d = wi ^ wj;
                        if (lim < 32) d &= (uint64_t(1) << (2 * lim)) - 1;
                    }
                    if (d) {
                        h = (__ffsll((long long)d) - 1) >> 1;
                    } else {
                        h = listed ? lcp_listed(t, T.P, lst, nexc, n32, i, j, lim, kLcpCap, keep)
                                   : lcp_bitmap(t, T, n32, i, j, 0, kLcpCap);
                        if (h >= kLcpCap) {
                            const uint32_t slot = atomicAdd(reinterpret_cast<unsigned *>(&T.ctl[kCtlLong]), 1u);
                            if (slot < uint32_t(n)) longl[slot] = uint32_t(k);
                        }
                    }
                }
            }
            st_i32_hint(lcp + k, h, once);
        }
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
}

// The listed ranks' LCP from kLcpCap on, up to kLcpBudget symbols.  More
// listed ranks than `max_long`, or a comparison that reaches the budget,
// sets the fallback flag (and leaves LCP to the Kasai passes).
__global__ void k_lcp_long(const uint8_t *__restrict__ t, PackedText T, int64_t n, const int32_t *__restrict__ sa,
                           int32_t *__restrict__ lcp, const uint32_t *__restrict__ longl, int64_t max_long) {
    const int64_t cnt = int64_t(uint32_t(T.ctl[kCtlLong]));
    if (cnt > max_long) {
        if (blockIdx.x == 0 && threadIdx.x == 0) T.ctl[kCtlFallback] = 1;
        return;
    }
    const int nexc = T.ctl[1];
    const bool listed = nexc <= kExcCap;
    const uint64_t keep = l2_policy_evict_last();
    const int32_t n32 = int32_t(n);
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < cnt; e += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t k = longl[e];
        const int32_t i = sa[k], j = sa[k - 1];  // both checked by k_lcp_direct
        const int32_t h = listed ? lcp_listed(t, T.P, T.list, nexc, n32, i, j, kLcpCap, kLcpBudget, keep)
                                 : lcp_bitmap(t, T, n32, i, j, kLcpCap, kLcpBudget);
        if (h >= kLcpBudget) T.ctl[kCtlFallback] = 1;
        else lcp[k] = h;
    }
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
