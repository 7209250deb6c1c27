// abi.cu -- status reporting, launch accounting, kernel timing and the
// standalone radix-sort entry point of liblor.
#include <atomic>
#include <mutex>
#include <vector>

#include "radix.cuh"

LOR_DEFINE_TU_STATUS(lor_status_abi)

namespace lor {

static std::atomic<unsigned long long> g_launches{0};
// While a thread captures work into a CUDA graph its launches are counted
// apart (they run when the graph is launched, as often as it is launched).
static thread_local bool t_capturing = false;
static thread_local unsigned long long t_captured = 0;
void note_launch() {
    if (t_capturing) ++t_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void capture_begin() {
    t_capturing = true;
    t_captured = 0;
}
unsigned long long capture_end() {
    t_capturing = false;
    return t_captured;
}
void note_graph_launches(unsigned long long kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }

static thread_local int *t_status_slot = nullptr;
int *status_slot() { return t_status_slot; }
void set_status_slot(int *d_slot) { t_status_slot = d_slot; }
int read_status_slot(int *d_slot, cudaStream_t s) {
    int h = 0;
    LOR_CUDA_TRY(cudaMemcpyAsync(&h, d_slot, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaStreamSynchronize(s));
    if (h != 0) {
        LOR_CUDA_TRY(cudaMemsetAsync(d_slot, 0, sizeof(int), s));
        LOR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return h;
}

// ---------------------------------------------------------------- timing

namespace {
struct ProfRec {
    int kind;
    double bytes;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

const char *kKindNames[PK_COUNT] = {
    "encode", "sample_keys", "radix_hist", "radix_pass", "naming", "rank_scatter", "nonsample",
    "merge", "isa_scatter", "kasai", "overlap_scan", "overlap_collect", "rmq_level", "rmq_query",
    "other"};
}  // namespace

bool prof_enabled() { return g_prof_on; }

// ---------------------------------------------------------------- launch parameters

namespace {
std::mutex g_tune_mu;
TuneConfig g_tune;
}  // namespace

TuneConfig tune_config() {
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_tune;
}

static bool tune_valid(const lor_tune &c) {
    return c.digit_bits >= 5 && c.digit_bits <= 8 && c.level0_key_bits >= 24 && c.level0_key_bits <= 60 &&
           (c.sort_items_64 == 8 || c.sort_items_64 == 12 || c.sort_items_64 == 16) && (c.sort_items_32 == 12 || c.sort_items_32 == 16) &&
           (c.merge_items == 2 || c.merge_items == 4 || c.merge_items == 8);
}

ProfScope::ProfScope(int kind, double bytes, cudaStream_t s) : stream(s) {
    if (!g_prof_on || t_capturing) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    ProfRec r;
    r.kind = kind;
    r.bytes = bytes;
    r.a = take_event();
    r.b = take_event();
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    slot = int(g_recs.size()) - 1;
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    cudaEventRecord(g_recs[slot].b, stream);
}

}  // namespace lor

using namespace lor;

extern "C" uint64_t lor_launch_count(void) { return g_launches.load(); }

extern "C" int lor_profile_enable(int on) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = on != 0;
    while (g_prof_on && g_pool.size() < 512) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return LOR_ERR_CUDA;
        g_pool.push_back(e);
    }
    return LOR_OK;
}

extern "C" int lor_profile_reset(void) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return LOR_OK;
}

extern "C" int lor_profile_kinds(void) { return PK_COUNT; }

extern "C" const char *lor_profile_kind_name(int kind) {
    return (kind >= 0 && kind < PK_COUNT) ? kKindNames[kind] : "unknown";
}

extern "C" int lor_profile_read(int kind, int64_t *h_launches, double *h_ms, double *h_bytes) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    int64_t cnt = 0;
    double ms = 0, bytes = 0;
    for (auto &r : g_recs) {
        if (r.kind != kind) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return LOR_ERR_CUDA;
        float t = 0;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return LOR_ERR_CUDA;
        cnt++;
        ms += t;
        bytes += r.bytes;
    }
    if (h_launches) *h_launches = cnt;
    if (h_ms) *h_ms = ms;
    if (h_bytes) *h_bytes = bytes;
    return LOR_OK;
}

// ---------------------------------------------------------------- status

extern "C" int lor_device_status(lor_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LOR_ERR_CUDA;
    int first = LOR_OK;
    int (*fns[])(cudaStream_t, int) = {lor_status_encode, lor_status_dc3, lor_status_lcp,
                                       lor_status_overlap, lor_status_rmq, lor_status_abi,
                                       lor_status_batch, lor_status_serve, lor_status_multi,
                                       lor_status_topk, lor_status_sa64};
    for (auto f : fns) {
        const int v = f(s, 1);
        if (v != LOR_OK && first == LOR_OK) first = v;
    }
    return first;
}

extern "C" int lor_test_set_wait(uint64_t limit_ns, int32_t starve_first_tile) {
    if (starve_first_tile != 0 && starve_first_tile != 1) return LOR_ERR_INVALID_ARG;
    const uint64_t lim = limit_ns ? limit_ns : kSpinLimitNs;
    if (lim > kSpinLimitNs) return LOR_ERR_INVALID_ARG;
    int (*fns[])(uint64_t, int) = {lor_status_encode_set_wait, lor_status_dc3_set_wait, lor_status_lcp_set_wait,
                                   lor_status_overlap_set_wait, lor_status_rmq_set_wait, lor_status_abi_set_wait,
                                   lor_status_batch_set_wait, lor_status_serve_set_wait, lor_status_multi_set_wait,
                                   lor_status_topk_set_wait, lor_status_sa64_set_wait};
    for (auto f : fns) {
        const int rc = f(lim, starve_first_tile);
        if (rc != LOR_OK) return rc;
    }
    return LOR_OK;
}

extern "C" const char *lor_status_string(int status) {
    switch (status) {
        case LOR_OK: return "ok";
        case LOR_ERR_INVALID_ARG: return "invalid argument";
        case LOR_ERR_BAD_SYMBOL: return "symbol outside the alphabet";
        case LOR_ERR_TOO_LARGE: return "text longer than LOR_MAX_N";
        case LOR_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case LOR_ERR_CUDA: return "CUDA runtime error";
        case LOR_ERR_TIMEOUT: return "bounded device wait expired";
        case LOR_ERR_BAD_INPUT: return "input array holds an out-of-range index";
        case LOR_ERR_CANCELLED: return "server shut down before the request ran";
        default: return "unknown status";
    }
}

// ---------------------------------------------------------------- radix sort

namespace {
struct SortLayout {
    size_t ctrl = 0, hist = 0, offsets = 0, lookback = 0, lookback_bytes = 0, kb = 0, vb = 0, total = 0;
};
SortLayout sort_layout(int64_t m) {
    SortLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.ctrl = take(256);
    L.hist = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.offsets = take(sizeof(uint32_t) * kMaxPasses * kRadix);
    L.lookback_bytes = radix_lookback_bytes(m);
    L.lookback = take(L.lookback_bytes);
    L.kb = take(sizeof(uint64_t) * size_t(m));
    L.vb = take(sizeof(uint32_t) * size_t(m));
    L.total = off;
    return L;
}
}  // namespace

extern "C" size_t lor_radix_sort_workspace_size(int64_t m) {
    if (m < 0 || m > LOR_MAX_N) return 0;
    return sort_layout(m).total;
}

extern "C" int lor_radix_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, int64_t m, int32_t key_bits,
                                    void *d_ws, size_t ws_bytes, lor_stream_t stream) {
    if (m < 0 || key_bits < 0 || key_bits > 64) return LOR_ERR_INVALID_ARG;
    if (m == 0) return LOR_OK;
    if (!d_keys || !d_vals) return LOR_ERR_INVALID_ARG;
    if (m > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const SortLayout L = sort_layout(m);
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
    rs.max_tiles = cdiv(m, kMinSortTile);
    rs.status = status;
    rs.stream = s;
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, 256, s));
    LOR_CUDA_TRY(cudaMemsetAsync(ws + L.lookback, 0, L.lookback_bytes, s));
    uint64_t *kb = (uint64_t *)(ws + L.kb);
    uint32_t *vb = (uint32_t *)(ws + L.vb);
    uint64_t *kr;
    uint32_t *vr;
    const int rc = radix_sort_pairs<uint64_t>(rs, d_keys, d_vals, kb, vb, m, 0, key_bits, false, &kr, &vr);
    if (rc) return rc;
    if (kr != d_keys) {
        LOR_CUDA_TRY(cudaMemcpyAsync(d_keys, kr, sizeof(uint64_t) * size_t(m), cudaMemcpyDeviceToDevice, s));
        LOR_CUDA_TRY(cudaMemcpyAsync(d_vals, vr, sizeof(uint32_t) * size_t(m), cudaMemcpyDeviceToDevice, s));
    }
    return LOR_OK;
}

extern "C" void lor_tune_default(lor_tune *cfg) {
    if (!cfg) return;
    const TuneConfig d;
    cfg->digit_bits = d.digit_bits;
    cfg->level0_key_bits = d.level0_key_bits;
    cfg->sort_items_64 = d.sort_items_64;
    cfg->sort_items_32 = d.sort_items_32;
    cfg->merge_items = d.merge_items;
}

extern "C" int lor_tune_get(lor_tune *cfg) {
    if (!cfg) return LOR_ERR_INVALID_ARG;
    const TuneConfig c = tune_config();
    cfg->digit_bits = c.digit_bits;
    cfg->level0_key_bits = c.level0_key_bits;
    cfg->sort_items_64 = c.sort_items_64;
    cfg->sort_items_32 = c.sort_items_32;
    cfg->merge_items = c.merge_items;
    return LOR_OK;
}

extern "C" int lor_tune_set(const lor_tune *cfg) {
    if (!cfg || !tune_valid(*cfg)) return LOR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.digit_bits = cfg->digit_bits;
    g_tune.level0_key_bits = cfg->level0_key_bits;
    g_tune.sort_items_64 = cfg->sort_items_64;
    g_tune.sort_items_32 = cfg->sort_items_32;
    g_tune.merge_items = cfg->merge_items;
    return LOR_OK;
}
