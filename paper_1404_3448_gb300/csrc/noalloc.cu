// noalloc.cu -- suffix array for callers that cannot allocate device memory.
//
// lor_build_sa needs a caller-provided workspace of about 60 bytes per text
// symbol.  Some callers cannot call cudaMalloc (or any allocating routine) at
// the point where they need a suffix array: a plugin running inside a host
// application that owns the device memory pool, a callback that must not
// block on or fragment the allocator, or code in a process whose allocator is
// locked down.  lor_build_sa_noalloc serves them for texts of up to
// LOR_NOALLOC_MAX_N symbols: its scratch is one file-scope device array that
// is part of the library image, so the call itself allocates nothing.
//
// The array is created on every GPU that loads the library and stays there
// until the process exits.  All calls share it, so calls whose GPU work can
// overlap (different streams, different host threads) race on it and must be
// serialised by the caller.  lor_build_sa clears the parts that must start at
// zero (counters and look-back flags) at the start of every call, so the
// contents left by the previous call do no harm.
//
// The array's device address is looked up once per device and kept for the
// life of the process; after cudaDeviceReset the library's device memory is
// gone (the array may come back elsewhere), so this entry point must not be
// used again in that process.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LOR_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LOR_ERR_CUDA;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return LOR_OK;
}

}  // namespace

extern "C" int lor_build_sa_noalloc(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa,
                                    lor_stream_t stream) {
    // argument checks in lor_build_sa's order, then this entry point's size limit
    if (!d_text || !d_sa || n < 1 || sigma < 2 || sigma > 256) return LOR_ERR_INVALID_ARG;
    if (n > LOR_NOALLOC_MAX_N) return LOR_ERR_TOO_LARGE;
    const size_t need = lor_build_sa_workspace_size(n, sigma);
    if (need == 0 || need > kNoAllocScratchBytes) return LOR_ERR_WORKSPACE;
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != LOR_OK) return rc;
    return lor_build_sa(d_text, n, sigma, d_sa, ws, kNoAllocScratchBytes, stream);
}
