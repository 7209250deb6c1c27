// encode.cu -- ASCII DNA to symbol codes, concatenated with one unique
// terminator per sequence (Section 3: the overlap of two sequences is read
// from one suffix array over both; the separator scheme is this library's
// reading).  Terminator of sequence i = nseq - i, A/C/G/T = nseq+1..nseq+4,
// so the last terminator is the smallest symbol and A < C < G < T as in
// Table 1.
#include "common.cuh"

LOR_DEFINE_TU_STATUS(lor_status_encode)

namespace lor {
namespace {

struct EncParams {
    int32_t nseq;
    int64_t n_ascii;  // bytes of the ASCII input (the sum of the lengths)
    int64_t out_start[LOR_MAX_SEQ + 1];  // start of sequence i in the text; [nseq] = n
};

constexpr int kEncThreads = 256;
constexpr int kEncItems = 16;  // bytes per thread

template <typename StT>
__global__ void __launch_bounds__(kEncThreads) k_encode(const uint8_t *__restrict__ ascii, EncParams P,
                                                        uint8_t *__restrict__ text, int64_t n,
                                                        StT *__restrict__ starts, int *status) {
    __shared__ int64_t so[LOR_MAX_SEQ + 1];
    __shared__ uint8_t lut[256];
    const int nseq = P.nseq;
    for (int i = threadIdx.x; i <= nseq; i += blockDim.x) so[i] = P.out_start[i];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
        uint8_t v = 0;
        if (c == 'A' || c == 'a') v = uint8_t(nseq + 1);
        if (c == 'C' || c == 'c') v = uint8_t(nseq + 2);
        if (c == 'G' || c == 'g') v = uint8_t(nseq + 3);
        if (c == 'T' || c == 't') v = uint8_t(nseq + 4);
        lut[c] = v;
    }
    __syncthreads();
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (starts && gid <= nseq) starts[gid] = StT(so[gid]);
    const int64_t o0 = gid * kEncItems;
    if (o0 >= n) return;
    // sequence holding o0
    int lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (so[mid] <= o0) lo = mid;
        else hi = mid - 1;
    }
    int sq = lo;
    bool bad = false;
    // The 16 codes are assembled in registers and stored with one 16-byte
    // write when the run is whole and aligned (byte stores from lanes 16
    // bytes apart would each touch a separate sector).
    uint32_t w[kEncItems / 4] = {0, 0, 0, 0};
    // A run inside one sequence's bases reads its 16 source bytes with two
    // aligned 16-byte loads (the source is offset by the terminators before
    // it) and picks them out with byte permutes.
    const int64_t src = o0 - sq, a0 = src & ~int64_t(15);
    if (o0 + kEncItems < so[sq + 1] && ((uintptr_t)ascii & 15) == 0 && a0 + 32 <= P.n_ascii) {
        const uint4 u = *reinterpret_cast<const uint4 *>(ascii + a0);
        const uint4 v = *reinterpret_cast<const uint4 *>(ascii + a0 + 16);
        const uint32_t x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
        const int r = int(src - a0);  // bytes to skip, 0..15
#pragma unroll
        for (int c = 0; c < kEncItems / 4; ++c) {
            // the four source bytes r + 4c .. r + 4c + 3 of the 32 loaded
            const int b = r + 4 * c, wi = b >> 2, sh = b & 3;
            uint32_t lo4 = x[0], hi4 = x[1];
#pragma unroll
            for (int q = 1; q < 7; ++q)
                if (wi == q) {
                    lo4 = x[q];
                    hi4 = x[q + 1];
                }
            const uint32_t bytes = __byte_perm(lo4, hi4, uint32_t(0x3210 + 0x1111 * sh));
            uint32_t out = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t code = lut[(bytes >> (8 * e)) & 0xFFu];
                if (code == 0) {
                    bad = true;
                    code = uint32_t(nseq + 1);
                }
                out |= code << (8 * e);
            }
            w[c] = out;
        }
    } else {
#pragma unroll
    for (int k = 0; k < kEncItems; ++k) {
        const int64_t o = o0 + k;
        if (o >= n) break;
        while (o >= so[sq + 1]) ++sq;
        const int64_t term = so[sq + 1] - 1;
        uint32_t v;
        if (o == term) {
            v = uint32_t(nseq - sq);
        } else {
            v = lut[ascii[o - sq]];
            if (v == 0) {
                bad = true;
                v = uint32_t(nseq + 1);
            }
        }
        w[k >> 2] |= v << (8 * (k & 3));
    }
    }
    if (o0 + kEncItems <= n && ((uintptr_t(text + o0) & 15) == 0)) {
        *reinterpret_cast<uint4 *>(text + o0) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
        for (int k = 0; k < kEncItems && o0 + k < n; ++k) text[o0 + k] = uint8_t(w[k >> 2] >> (8 * (k & 3)));
    }
    if (bad) atomicCAS(status, 0, LOR_ERR_BAD_SYMBOL);
}

}  // namespace
}  // namespace lor

using namespace lor;

namespace lor {
namespace {

template <typename StT>
int encode_impl(const uint8_t *d_ascii, const int64_t *h_lens, int32_t nseq, uint8_t *d_text, StT *d_seq_starts,
                lor_stream_t stream, int64_t max_n) {
    if (nseq < 1 || nseq > LOR_MAX_SEQ || !h_lens || !d_text) return LOR_ERR_INVALID_ARG;
    EncParams P;
    P.nseq = nseq;
    int64_t total = 0;
    for (int i = 0; i < nseq; ++i) {
        if (h_lens[i] < 0) return LOR_ERR_INVALID_ARG;
        P.out_start[i] = total;
        total += h_lens[i] + 1;
        if (total > max_n) return LOR_ERR_TOO_LARGE;
    }
    P.out_start[nseq] = total;
    P.n_ascii = total - nseq;
    if (total > nseq && !d_ascii) return LOR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = tu_status_ptr();
    if (!status) return LOR_ERR_CUDA;
    const int64_t threads = cdiv(total, kEncItems) > nseq + 1 ? cdiv(total, kEncItems) : nseq + 1;
    {
        ProfScope ps(PK_ENCODE, double(total) * 2, s);
        k_encode<StT><<<unsigned(cdiv(threads, kEncThreads)), kEncThreads, 0, s>>>(d_ascii, P, d_text, total,
                                                                               d_seq_starts, status);
    }
    LOR_LAUNCH_CHECK();
    return LOR_OK;
}

}  // namespace
}  // namespace lor

extern "C" int lor_encode_concat(const uint8_t *d_ascii, const int64_t *h_lens, int32_t nseq, uint8_t *d_text,
                                 int32_t *d_seq_starts, lor_stream_t stream) {
    return encode_impl(d_ascii, h_lens, nseq, d_text, d_seq_starts, stream, LOR_MAX_N);
}

extern "C" int lor_encode_concat64(const uint8_t *d_ascii, const int64_t *h_lens, int32_t nseq, uint8_t *d_text,
                                   int64_t *d_seq_starts, lor_stream_t stream) {
    return encode_impl(d_ascii, h_lens, nseq, d_text, d_seq_starts, stream, LOR_MAX_N64);
}
