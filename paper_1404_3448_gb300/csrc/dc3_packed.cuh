// dc3_packed.cuh -- level-0 sample keys of DNA texts: 16 symbols at 2 bits.
//
// Step 1 of DC3 (Section 3) may name each sample by any prefix of its suffix
// at least three symbols long: the order of the reduced string's suffixes is
// then still the order of the sample suffixes.  For a text whose symbols are
// (apart from a few) the four largest codes -- DNA with its separators --
// the prefix of 16 symbols fits 32 bits at 2 bits a symbol.  A window that
// meets a smaller code (a separator, or the padding past the end) is an
// "exception": its key holds the symbols before that code and zeros after
// it, and a 33rd bit, below the key, puts it ahead of the ordinary window of
// the same 32 bits (the smaller code sorts before every base).  Exception
// windows whose 32 bits are equal are put in order afterwards by one block
// that compares their symbols (there are at most kPkExcMax of them; more and
// the level falls back to keys in base maxc + 1).
//
// The sort is LSD: the first pass partitions by the exception bit and the
// low key byte (512 buckets, not stable: equal keys get one name and nothing
// reads their order) and generates the keys from the text as it goes, so no
// key array is written before it; three stable 8-bit passes follow on
// (u32 key, u32 value) pairs.  The value is the sample index with the
// exception bit in bit 31.
#pragma once

#include "radix.cuh"
#include "scan.cuh"

namespace lor {

constexpr int kPkChars = 16;                          // symbols named by a key
constexpr int kPkTile = 4096;                         // samples per tile (one residue class)
constexpr int kPkThreads = 256;
constexpr int kPkItems = kPkTile / kPkThreads;        // 16
constexpr int kPkDigits0 = 512;                       // first pass: exception bit + low key byte
constexpr int kPkExcMax = 4096;                       // exception windows the fix-up can order
constexpr int kPkWords = (3 * kPkTile + 32) / 16 + 3; // 16-symbol words of a staged tile
// Histogram layout (u32 words): passes 1..3 at [0, 768), pass 0's 512 bins
// at [768, 1280), then the number of exception windows.
constexpr int kPkHist0 = 3 * kRadix;
constexpr int kPkExcCount = kPkHist0 + kPkDigits0;
constexpr int kPkHistWords = kPkExcCount + 1;

// The text of one tile, 16 symbols a word: 2-bit values (code - lo for the
// four largest codes, most significant first) and a 16-bit mask of the
// positions holding a smaller code (bit 15 = the word's first position).
struct PkText {
    uint32_t v[kPkWords];
    uint32_t e[kPkWords];
};

// Four text bytes (little-endian, first symbol in the low byte), every byte
// below 128 and lo <= 128, to their 2-bit values (8 bits, first symbol most
// significant) and exception nibble.  With the top bit of each byte set
// first, subtracting lo from every byte borrows across no byte boundary: the
// top bit survives exactly where the byte is at least lo, and the low two
// bits are those of byte - lo (128 is a multiple of 4).
__device__ __forceinline__ void pk_pack4(uint32_t x, uint32_t lo4, uint32_t &val8, uint32_t &exc4) {
    const uint32_t d = (x | 0x80808080u) - lo4;
    const uint32_t ge = (d >> 7) & 0x01010101u;  // 1 in each byte >= lo
    const uint32_t y = d & (ge * 3u);
    // gathers the four 2-bit fields b0..b3 into b0 b1 b2 b3 (no carries: the
    // other products land on distinct bits below 24 or above 31)
    val8 = (y * 0x40100401u) >> 24;
    exc4 = (((ge ^ 0x01010101u)) * 0x08040201u) >> 24;
}

// Any byte of x outside [1, maxc] (x's bytes below 128, maxc < 128).
__device__ __forceinline__ bool pk_out_of_range4(uint32_t x, uint32_t above4) {
    const uint32_t zero = (x - 0x01010101u) & ~x & 0x80808080u;
    const uint32_t high = ((x | 0x80808080u) - above4) & 0x80808080u;  // bytes >= maxc + 1
    return (zero | high | (x & 0x80808080u)) != 0;
}

// Stages text positions [a0, a0 + 16 * nwords) as PkText (positions >= n
// read as the padding 0, an exception).  Codes outside [1, maxc] are
// reported through *bad and clamped, as the other key makers do.
__device__ __forceinline__ void pk_stage(const uint8_t *__restrict__ s, int64_t n, uint32_t maxc, uint32_t lo,
                                         int64_t a0, int nwords, PkText &T, bool &bad) {
    const uint32_t lo4 = lo * 0x01010101u, above4 = (maxc + 1) * 0x01010101u;
    const bool vec = ((uintptr_t)s & 15) == 0 && maxc < 128;
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
        const int64_t q = a0 + 16 * int64_t(w);
        uint32_t x[4];
        bool slow = !(vec && q + 16 <= n);
        if (!slow) {
            const uint4 u = *reinterpret_cast<const uint4 *>(s + q);
            x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
            slow = pk_out_of_range4(x[0], above4) || pk_out_of_range4(x[1], above4) ||
                   pk_out_of_range4(x[2], above4) || pk_out_of_range4(x[3], above4);
        }
        if (slow) {  // the text's end, an unaligned text, large codes or codes to clamp
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t t = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int64_t p = q + 4 * c + b;
                    uint32_t code = 0;  // the padding past the end
                    if (p < n) {
                        code = s[p];
                        if (code < 1 || code > maxc) {
                            bad = true;
                            code = code < 1 ? 1u : maxc;
                        }
                    }
                    // as a 2-bit value (bit 7 clear) or an exception (bit 7 set)
                    t |= (code >= lo ? (code - lo) : 0x80u) << (8 * b);
                }
                x[c] = t;
            }
        }
        uint32_t val = 0, exc = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t v8, e4;
            if (slow) {  // bytes already mapped: the 2-bit value, or bit 7 for an exception
                const uint32_t e = (x[c] >> 7) & 0x01010101u;
                v8 = ((x[c] & 0x03030303u) * 0x40100401u) >> 24;
                e4 = (e * 0x08040201u) >> 24;
            } else {
                pk_pack4(x[c], lo4, v8, e4);
            }
            val |= v8 << (24 - 8 * c);
            exc |= e4 << (12 - 4 * c);
        }
        T.v[w] = val;
        T.e[w] = exc;
    }
}

// The key of the window at staged position q: its 16 symbols' 2-bit values
// with everything from the first exception on cleared; *exc set when the
// window holds an exception.
__device__ __forceinline__ uint32_t pk_window(const PkText &T, int q, bool &exc) {
    const int w = q >> 4, r = q & 15;
    uint32_t key = __funnelshift_l(T.v[w + 1], T.v[w], 2 * r);
    const uint32_t em = (((T.e[w] << 16) | T.e[w + 1]) << r) & 0xFFFF0000u;
    exc = em != 0;
    if (exc) {
        const int jx = __clz(em);  // offset of the first exception
        key = jx ? key & (~0u << (32 - 2 * jx)) : 0u;
    }
    return key;
}

__device__ __forceinline__ uint32_t pk_digit0(uint32_t key, bool exc) { return ((key & 0xFFu) << 1) | (exc ? 0u : 1u); }

// The clamped code at text position p (0 past the end), as the key makers
// read it.
__device__ __forceinline__ uint32_t pk_code(const uint8_t *__restrict__ s, int64_t n, int64_t p, uint32_t maxc) {
    if (p >= n) return 0;
    const uint32_t c = s[p];
    return c < 1 ? 1u : (c > maxc ? maxc : c);
}

// Staged span of a tile: its first position rounded down to 16, and words.
__device__ __forceinline__ void pk_tile_span(int64_t j0, int cls, int nj, int64_t &a0, int &off, int &nwords) {
    const int64_t p0 = 3 * j0 + 1 + cls;
    a0 = p0 & ~int64_t(15);
    off = int(p0 - a0);
    nwords = ((off + 3 * (nj - 1)) >> 4) + 2;
}

// Pre-pass: the four passes' digit histograms and the list of exception
// windows (sample indices; only the first kPkExcMax are kept, the count is
// exact).  Block (x, c): kPkTile samples of class c (c = 0: positions 3j+1,
// stored at j; c = 1: positions 3j+2, stored at n0 + j).
static __global__ void __launch_bounds__(kPkThreads) k_pk_count(const uint8_t *__restrict__ s, int64_t n, int64_t n0,
                                                         int64_t n2, uint32_t maxc, uint32_t lo,
                                                         uint32_t *__restrict__ hist, uint32_t *__restrict__ exc_list,
                                                         int *status) {
    __shared__ PkText T;
    __shared__ uint32_t h[kPkHistWords - 1];
    const int tid = threadIdx.x;
    const int cls = int(blockIdx.y);
    const int64_t ncls = cls == 0 ? n0 : n2;
    const int64_t j0 = int64_t(blockIdx.x) * kPkTile;
    if (j0 >= ncls) return;  // uniform over the block
    const int nj = int(min64(int64_t(kPkTile), ncls - j0));
    int64_t a0;
    int off, nwords;
    pk_tile_span(j0, cls, nj, a0, off, nwords);
    bool bad = false;
    pk_stage(s, n, maxc, lo, a0, nwords, T, bad);
    for (int i = tid; i < kPkHistWords - 1; i += kPkThreads) h[i] = 0;
    __syncthreads();
    const int64_t jbase = (cls == 0 ? 0 : n0) + j0;
    for (int i = 0; i < kPkItems; ++i) {
        const int k = i * kPkThreads + tid;
        const bool valid = k < nj;
        bool exc = false;
        const uint32_t key = valid ? pk_window(T, off + 3 * k, exc) : 0u;
        const uint32_t d0 = pk_digit0(key, exc);
        // a warp whose 32 windows share one key counts it once, by 32 (texts
        // of one repeated symbol would otherwise serialise on one counter)
        const uint32_t k0 = __shfl_sync(0xffffffffu, key, 0), x0 = __shfl_sync(0xffffffffu, uint32_t(exc), 0);
        if (__all_sync(0xffffffffu, valid && key == k0 && uint32_t(exc) == x0)) {
            if ((tid & 31) == 0) {
                atomicAdd(&h[kPkHist0 + d0], 32u);
                atomicAdd(&h[(key >> 8) & 0xFFu], 32u);
                atomicAdd(&h[kRadix + ((key >> 16) & 0xFFu)], 32u);
                atomicAdd(&h[2 * kRadix + (key >> 24)], 32u);
            }
        } else if (valid) {
            atomicAdd(&h[kPkHist0 + d0], 1u);
            atomicAdd(&h[(key >> 8) & 0xFFu], 1u);
            atomicAdd(&h[kRadix + ((key >> 16) & 0xFFu)], 1u);
            atomicAdd(&h[2 * kRadix + (key >> 24)], 1u);
        }
        if (exc) {
            const uint32_t slot = atomicAdd(&hist[kPkExcCount], 1u);
            if (slot < uint32_t(kPkExcMax)) exc_list[slot] = uint32_t(jbase + k);
        }
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
    __syncthreads();
    for (int i = tid; i < kPkHistWords - 1; i += kPkThreads)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Bucket starts: exclusive scans of passes 1..3 (256 bins each) into
// offsets[0, 768) and of pass 0 (512 bins) into offsets[768, 1280).
static __global__ void __launch_bounds__(kRadix) k_pk_offsets(const uint32_t *__restrict__ hist, uint32_t *__restrict__ offsets) {
    __shared__ uint32_t scratch[kRadix / 32 + 1];
    const int t = threadIdx.x;
    uint32_t total;
    for (int p = 0; p < 3; ++p) offsets[p * kRadix + t] = block_excl_scan<kRadix>(hist[p * kRadix + t], scratch, &total);
    const uint32_t a = hist[kPkHist0 + 2 * t], b = hist[kPkHist0 + 2 * t + 1];
    const uint32_t x = block_excl_scan<kRadix>(a + b, scratch, &total);
    offsets[kPkHist0 + 2 * t] = x;
    offsets[kPkHist0 + 2 * t + 1] = x + a;
}

struct PkPartSmem {
    PkText T;
    uint32_t keys[kPkTile];
    uint32_t vals[kPkTile];
    uint32_t cnt[kPkDigits0];
    uint32_t local_start[kPkDigits0];
    long long gbase[kPkDigits0];
    uint32_t scratch[kPkThreads / 32 + 1];
};

// First pass: every tile makes its samples' keys from the text and
// partitions them by pk_digit0 into (kout, vout) without look-back (as
// k_partition: a shared-memory atomic places an element inside its tile's
// digit run; one global atomic per digit reserves the run in the bucket,
// cursor[d] starting at the bucket's offset).  Tiles are numbered class 0
// first; a persistent grid walks them with a grid stride.
static __global__ void __launch_bounds__(kPkThreads, 4) k_pk_partition(const uint8_t *__restrict__ s, int64_t n, int64_t n0,
                                                                int64_t n2, uint32_t maxc, uint32_t lo,
                                                                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                uint32_t *__restrict__ cursor, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PkPartSmem &S = *reinterpret_cast<PkPartSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t m = n0 + n2;
    const int64_t t0 = cdiv(n0, kPkTile), ntiles = t0 + cdiv(n2, kPkTile);
    bool bad = false;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int cls = tile < t0 ? 0 : 1;
        const int64_t j0 = (tile - (cls ? t0 : 0)) * kPkTile;
        const int nj = int(min64(int64_t(kPkTile), (cls ? n2 : n0) - j0));
        int64_t a0;
        int off, nwords;
        pk_tile_span(j0, cls, nj, a0, off, nwords);
        if (tid == 0) {
            // ask the L2 for the text of this block's next tile
            const int64_t nt = tile + gridDim.x;
            if (nt < ntiles) {
                const int ncls = nt < t0 ? 0 : 1;
                const int64_t nj0 = (nt - (ncls ? t0 : 0)) * kPkTile;
                const int64_t b = 3 * nj0 + 1 + ncls;
                prefetch_inside(s + b, s + min64(n, b + 3 * kPkTile + kPkChars));
            }
        }
        pk_stage(s, n, maxc, lo, a0, nwords, S.T, bad);
        S.cnt[tid] = 0;
        S.cnt[tid + kPkThreads] = 0;
        __syncthreads();
        const uint32_t jbase = uint32_t((cls ? n0 : 0) + j0);
        uint32_t key[kPkItems], r[kPkItems];
        uint32_t excm = 0;
#pragma unroll
        for (int i = 0; i < kPkItems; ++i) {
            const int k = i * kPkThreads + tid;
            bool exc = false;
            key[i] = k < nj ? pk_window(S.T, off + 3 * k, exc) : 0u;
            excm |= uint32_t(exc) << i;
            r[i] = k < nj ? atomicAdd(&S.cnt[pk_digit0(key[i], exc)], 1u) : 0u;
        }
        __syncthreads();
        // thread t owns digits 2t and 2t + 1: their runs in the buckets and
        // their starts inside the tile
        const uint32_t ca = S.cnt[2 * tid], cb = S.cnt[2 * tid + 1];
        const uint32_t ra = ca ? atomicAdd(&cursor[2 * tid], ca) : 0u;
        const uint32_t rb = cb ? atomicAdd(&cursor[2 * tid + 1], cb) : 0u;
        uint32_t tile_total;
        const uint32_t ls = block_excl_scan<kPkThreads>(ca + cb, S.scratch, &tile_total);
        S.local_start[2 * tid] = ls;
        S.local_start[2 * tid + 1] = ls + ca;
        S.gbase[2 * tid] = (long long)ra - ls;
        S.gbase[2 * tid + 1] = (long long)rb - (ls + ca);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kPkItems; ++i) {
            const int k = i * kPkThreads + tid;
            if (k < nj) {
                const bool exc = (excm >> i) & 1u;
                const uint32_t pos = S.local_start[pk_digit0(key[i], exc)] + r[i];
                S.keys[pos] = key[i];
                S.vals[pos] = (jbase + uint32_t(k)) | (exc ? 0x80000000u : 0u);
            }
        }
        __syncthreads();
        for (int i = tid; i < nj; i += kPkThreads) {
            const uint32_t kk = S.keys[i], vv = S.vals[i];
            const long long o = S.gbase[pk_digit0(kk, vv >> 31)] + i;
            if (o < 0 || o >= m) {  // counts that did not match the keys
                atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
                continue;
            }
            kout[o] = kk;
            vout[o] = vv;
        }
        __syncthreads();  // staging and counts are reused by the next tile
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
}

// ---- ordering the exception windows that share their 32 key bits

struct PkFixSmem {
    uint32_t key[kPkExcMax];      // the 32 key bits
    uint32_t tail[kPkExcMax][4];  // symbols from the first exception on, big-endian bytes
    uint32_t j[kPkExcMax];        // sample index
    uint8_t jx[kPkExcMax];        // offset of the first exception
    uint16_t idx[kPkExcMax];      // sort order
};

__device__ __forceinline__ bool pk_fix_less(const PkFixSmem &F, int a, int b, int e) {
    if (b >= e) return a < e;  // entries past the count sort last
    if (a >= e) return false;
    if (F.key[a] != F.key[b]) return F.key[a] < F.key[b];
    if (F.jx[a] != F.jx[b]) return F.jx[a] < F.jx[b];
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (F.tail[a][w] != F.tail[b][w]) return F.tail[a][w] < F.tail[b][w];
    return false;
}

// Within the keys' sorted order, the exception windows of one 32-bit key k
// are the first entries of k's run (the exception bit sorted them ahead of
// the ordinary windows); here they are put in the order of their symbols:
// the earlier exception first (a smaller code against a base), then the
// symbols from the exception on.  One block; e <= kPkExcMax entries.
static __global__ void __launch_bounds__(1024) k_pk_fixup(const uint8_t *__restrict__ s, int64_t n, int64_t n0,
                                                   uint32_t maxc, uint32_t lo, const uint32_t *__restrict__ hist,
                                                   const uint32_t *__restrict__ exc_list,
                                                   const uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                   int64_t m, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PkFixSmem &F = *reinterpret_cast<PkFixSmem *>(smem_raw);
    const int e = int(min64(int64_t(hist[kPkExcCount]), int64_t(kPkExcMax)));
    if (e == 0) return;
    int np = 1;
    while (np < e) np <<= 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        F.idx[i] = uint16_t(i);
        if (i >= e) continue;
        const uint32_t j = exc_list[i];
        const int64_t p = j < n0 ? 3 * int64_t(j) + 1 : 3 * (int64_t(j) - n0) + 2;
        uint32_t w[kPkChars];
        int jx = kPkChars;
        uint32_t key = 0;
        for (int t = 0; t < kPkChars; ++t) {
            w[t] = pk_code(s, n, p + t, maxc);
            if (jx == kPkChars && w[t] < lo) jx = t;
            if (jx == kPkChars) key |= (w[t] - lo) << (30 - 2 * t);
        }
        uint32_t tl[4] = {0, 0, 0, 0};
        for (int t = jx; t < kPkChars; ++t) tl[(t - jx) >> 2] |= w[t] << (24 - 8 * ((t - jx) & 3));
        F.key[i] = key;
        F.jx[i] = uint8_t(jx);
        F.j[i] = j;
        for (int c = 0; c < 4; ++c) F.tail[i][c] = tl[c];
    }
    __syncthreads();
    // bitonic sort of the entry indices
    for (int size = 2; size <= np; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                const int partner = i ^ stride;
                if (partner > i) {
                    const bool up = (i & size) == 0;
                    const int a = F.idx[i], b = F.idx[partner];
                    const bool swap = up ? pk_fix_less(F, b, a, e) : pk_fix_less(F, a, b, e);
                    if (swap) {
                        F.idx[i] = uint16_t(b);
                        F.idx[partner] = uint16_t(a);
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < e; i += blockDim.x) {
        const int a = F.idx[i];
        const uint32_t k = F.key[a];
        // first entry of this key in the sorted list
        int lo_i = 0, hi_i = i;
        while (lo_i < hi_i) {
            const int mid = (lo_i + hi_i) >> 1;
            if (F.key[F.idx[mid]] < k) lo_i = mid + 1;
            else hi_i = mid;
        }
        // first slot of this key in the sorted keys
        int64_t lo_s = 0, hi_s = m;
        while (lo_s < hi_s) {
            const int64_t mid = (lo_s + hi_s) >> 1;
            if (keys[mid] < k) lo_s = mid + 1;
            else hi_s = mid;
        }
        const int64_t dst = lo_s + (i - lo_i);
        if (dst >= m || keys[dst] != k || !(vals[dst] >> 31)) {
            atomicCAS(status, 0, LOR_ERR_BAD_INPUT);  // the sort and the list disagree
            continue;
        }
        vals[dst] = F.j[a] | 0x80000000u;
    }
}

// Text position of sample j (class 0: 3j + 1; class 1: 3(j - n0) + 2).
__device__ __forceinline__ int64_t pk_sample_pos(uint32_t j, int64_t n0) {
    return int64_t(j) < n0 ? 3 * int64_t(j) + 1 : 3 * (int64_t(j) - n0) + 2;
}
// Two windows' 16 symbols, equal or not (exception windows of one key).
__device__ __forceinline__ bool pk_windows_equal(const uint8_t *__restrict__ s, int64_t n, int64_t n0, uint32_t maxc,
                                                 uint32_t ja, uint32_t jb) {
    const int64_t pa = pk_sample_pos(ja, n0), pb = pk_sample_pos(jb, n0);
    for (int t = 0; t < kPkChars; ++t)
        if (pk_code(s, n, pa + t, maxc) != pk_code(s, n, pb + t, maxc)) return false;
    return true;
}

// The 16 bytes from p as four big-endian words, read as five aligned
// 32-bit words (p + 20 <= n and s 4-byte aligned).
__device__ __forceinline__ void pk_load16_be(const uint8_t *__restrict__ s, int64_t p, uint32_t (&o)[4]) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(s + (p & ~int64_t(3)));
    const uint32_t r = uint32_t(p & 3);
    uint32_t x[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c] = w[c];
    // result byte 3 (most significant) = source byte r, ..., byte 0 = r + 3
    const uint32_t sel = (r + 3) | ((r + 2) << 4) | ((r + 1) << 8) | (r << 12);
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = __byte_perm(x[c], x[c + 1], sel);
}

// Order of the 16 symbols from p and from q (clamped codes, 0 past the
// end): -1, 0 or 1.  All 32 bytes are loaded before any is compared.  Away
// from the end of the text the raw bytes are compared (they differ from the
// clamped codes only at bad symbols, which are reported anyway).
__device__ __forceinline__ int pk_cmp16(const uint8_t *__restrict__ s, int64_t n, int64_t p, int64_t q, uint32_t maxc) {
    uint32_t a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
    if (((uintptr_t)s & 3) == 0 && p + 20 <= n && q + 20 <= n) {
        pk_load16_be(s, p, a);
        pk_load16_be(s, q, b);
    } else {
#pragma unroll
        for (int t = 0; t < kPkChars; ++t) {
            a[t >> 2] = (a[t >> 2] << 8) | pk_code(s, n, p + t, maxc);
            b[t >> 2] = (b[t >> 2] << 8) | pk_code(s, n, q + t, maxc);
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
    return 0;
}

// Naming of the sorted samples: a new name where the key, the exception bit
// or (between exception windows of one key) the symbols change.  Writes
// SA_R[j] = sample index, NS[j] = name, R[index] = name when R is given, the
// name count, and the positions j whose name is shared with a neighbour (the
// doubling's unresolved list, in order) with their names and count.  Each
// thread reads the entries on either side of its own sixteen.  Persistent, as
// k_name; the two counts share one block scan, and the two look-backs (names
// in lb, unresolved positions in lb2) run in warps 0 and 1.
static __global__ void __launch_bounds__(kScanThreads, 4) k_pk_name(const uint32_t *__restrict__ keys,
                                                                 const uint32_t *__restrict__ vals, int64_t m,
                                                                 const uint8_t *__restrict__ s, int64_t n, int64_t n0,
                                                                 uint32_t maxc, int32_t *__restrict__ R,
                                                                 int32_t *__restrict__ SAR, int32_t *__restrict__ NS,
                                                                 uint32_t *n_names, uint32_t *__restrict__ ul,
                                                                 int32_t *__restrict__ ul_names, uint32_t *ul_count,
                                                                 uint64_t *lb, uint64_t *lb2,
                                                                 unsigned long long *ctr, unsigned long long tile_base,
                                                                 uint32_t epoch, int *status) {
    constexpr int kW = kScanItems + 2;  // positions base-1 .. base+16
    __shared__ long long s_tile;
    __shared__ uint32_t scratch[kScanThreads / 32 + 1];
    __shared__ uint32_t s_prefix, s_uprefix;
    const int tid = threadIdx.x;
    const int64_t ntiles = cdiv(m > 0 ? m : 1, kScanTile);
    for (;;) {
        if (tid == 0) s_tile = (long long)(atomicAdd(ctr, 1ull) - tile_base);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;  // uniform over the block
        const int64_t base = tile * kScanTile + int64_t(tid) * kScanItems;
        uint32_t K[kW], V[kW];
        {
            uint32_t kk[kScanItems], vv[kScanItems];
            load_run<uint32_t, kScanItems>(keys, base, m, 0u, kk);
            load_run<uint32_t, kScanItems>(vals, base, m, 0u, vv);
#pragma unroll
            for (int i = 0; i < kScanItems; ++i) {
                K[i + 1] = kk[i];
                V[i + 1] = vv[i];
            }
            const bool lo_in = base >= 1 && base - 1 < m, hi_in = base + kScanItems < m;
            K[0] = lo_in ? keys[base - 1] : 0u;
            V[0] = lo_in ? vals[base - 1] : 0u;
            K[kW - 1] = hi_in ? keys[base + kScanItems] : 0u;
            V[kW - 1] = hi_in ? vals[base + kScanItems] : 0u;
        }
        // new-name bit x: position base-1+x differs from the one before it
        uint32_t newm = ~0u;
#pragma unroll
        for (int x = 1; x < kW; ++x) {
            const int64_t pos = base - 1 + x;
            if (pos >= 1 && pos < m) {
                bool same = K[x] == K[x - 1] && !((V[x] ^ V[x - 1]) >> 31);
                if (same && (V[x] >> 31))
                    same = pk_windows_equal(s, n, n0, maxc, V[x] & 0x7FFFFFFFu, V[x - 1] & 0x7FFFFFFFu);
                if (same) newm &= ~(1u << x);
            }
        }
        uint32_t flags = 0, cnt = 0, uflags = 0, ucnt = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int x = i + 1;
            const int64_t pos = base + i;
            if (pos < m) {
                const uint32_t f = (newm >> x) & 1u;
                flags |= f << i;
                cnt += f;
                const bool u = !f || (pos + 1 < m && !((newm >> (x + 1)) & 1u));
                uflags |= uint32_t(u) << i;
                ucnt += u;
            }
        }
        // both counts in one scan: each is at most kScanTile < 2^16 per tile
        uint32_t packed_agg;
        const uint32_t packed = block_excl_scan<kScanThreads>(cnt | (ucnt << 16), scratch, &packed_agg);
        const uint32_t excl = packed & 0xFFFFu, uexcl = packed >> 16;
        const uint32_t agg = packed_agg & 0xFFFFu, uagg = packed_agg >> 16;
        if (tid < 32) {
            const uint32_t p = warp_lookback(lb, tile, agg, epoch, status);
            if (tid == 0) s_prefix = p;
        } else if (tid < 64) {
            const uint32_t p = warp_lookback(lb2, tile, uagg, epoch, status);
            if (tid == 32) {
                s_uprefix = p;
                if (tile == ntiles - 1) *ul_count = p + uagg;
            }
        }
        __syncthreads();
        uint32_t name = s_prefix + excl, uo = s_uprefix + uexcl;
        int32_t nm[kScanItems], sa[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            name += (flags >> i) & 1u;
            nm[i] = int32_t(name);
            sa[i] = int32_t(V[i + 1] & 0x7FFFFFFFu);
            const int64_t pos = base + i;
            if (pos < m) {
                if (R) R[sa[i]] = int32_t(name);
                if (pos == m - 1) *n_names = name;
                if ((uflags >> i) & 1u) {
                    ul[uo] = uint32_t(pos);
                    ul_names[uo++] = int32_t(name);
                }
            }
        }
        store_run<int32_t, kScanItems>(SAR, base, m, sa);
        store_run<int32_t, kScanItems>(NS, base, m, nm);
        __syncthreads();  // s_tile and the prefixes are reused by the next tile
    }
}

// ---- the first round of the doubling at level 0, on the text itself

// Groups of exactly two samples that share their name (their first kchars
// symbols) are put in order by the next 16 symbols of the text, compared
// directly: their ranks become group head + 1 and + 2 (+ 1 for both when the
// symbols are equal too), so a pair is resolved without a rank round.  On
// text without long repeats almost every group is a pair.  Members of larger
// groups take the rank head + 1 (headof[name], when `headof` is given: the
// ranks were set to 1 + position before) and stay for the rank rounds.
// keep[i] marks list entries still unresolved.  One thread per entry of the
// ordered unresolved list ul, whose names come beside it (names[i]).
static __global__ void k_dbl_text_pairs(const uint32_t *__restrict__ ul, const int32_t *__restrict__ names,
                                        int64_t U,
                                        int32_t *__restrict__ SAR, int32_t *__restrict__ R,
                                        const int32_t *__restrict__ headof, const uint8_t *__restrict__ s,
                                        int64_t n, int64_t n0, uint32_t maxc, int kchars,
                                        uint32_t *__restrict__ keep) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < U; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t k = ul[i];
        const int32_t v = names[i];
        const bool start = i == 0 || names[i - 1] != v;
        const bool second = !start && (i < 2 || names[i - 2] != v);
        const bool pair = (start && (i + 2 >= U || names[i + 2] != v)) || (second && (i + 1 >= U || names[i + 1] != v));
        if (!pair) {
            if (headof) R[SAR[k]] = headof[v];
            keep[i] = 1u;
            continue;
        }
        if (!start) continue;  // the first member's thread settles the pair
        uint32_t a = uint32_t(SAR[k]), b = uint32_t(SAR[k + 1]);
        const int c = pk_cmp16(s, n, pk_sample_pos(a, n0) + kchars, pk_sample_pos(b, n0) + kchars, maxc);
        if (c > 0) {
            SAR[k] = int32_t(b);
            SAR[k + 1] = int32_t(a);
            const uint32_t t = a;
            a = b;
            b = t;
        }
        R[a] = int32_t(k + 1);
        R[b] = int32_t(c != 0 ? k + 2 : k + 1);
        keep[i] = keep[i + 1] = c == 0 ? 1u : 0u;
    }
}

}  // namespace lor
