// serve.cu -- request server over the grouped pipeline: pair requests arrive
// one at a time, free workers take the oldest waiting requests as one batch
// when the batch fits in the server's device reservation, and each request
// keeps its batch's ISA, LCP array and a linear-space (block) RMQ table over
// that LCP array on the device for LCP queries between arbitrary suffixes of
// its own text (Section 3: the LCP of two suffixes is the minimum of the
// adjacent LCPs between their ranks).
//
// Memory: one cudaMalloc of the whole budget at creation, managed by a
// first-fit allocator in 1 MiB granules.  A batch takes two blocks: its
// workspace (grouped-pipeline workspace, ASCII input, records, offsets and
// positions), returned as soon as the batch's results are on the host, and
// its resident state (ISA + LCP + block table, about 10.6 bytes per symbol
// where a full sparse table would need 4 + 4 * log2(n)), returned when the last of its
// requests is released.  A worker that cannot place the oldest waiting batch
// waits for memory to come back; requests are admitted in arrival order.
//
// Why results do not depend on the batching: block p of a batch's blocked
// suffix array is the suffix array of pair p's own text (see batch.cu), so
// ranks inside the block, the block's LCP values and the overlap record are
// those of the pair alone.  A query (p, q) of pair p reads ranks inside block
// p only: both ISA entries lie in the block, the partial 32-entry blocks at
// the ends of the range (r1, r2] are scanned inside it, and every window of
// whole blocks between them lies inside it, so the table rows need only
// bit_width(longest pair text / 32) levels and entries that span two pairs
// are never read.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "rmq_block.cuh"

LOR_DEFINE_TU_STATUS(lor_status_serve)

namespace lor {
namespace {

constexpr size_t kGranule = size_t(1) << 20;
constexpr size_t kNone = ~size_t(0);
constexpr int kQueryCap = 1 << 16;
constexpr int kMaxWorkers = 8;

size_t round_granule(size_t b) { return (b + kGranule - 1) & ~(kGranule - 1); }

// First-fit allocator over byte offsets [0, size) with coalescing.
class Arena {
  public:
    void init(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = peak_ = 0;
    }
    size_t alloc(size_t bytes) {
        bytes = round_granule(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[off + bytes] = rem;
            used_ += bytes;
            if (used_ > peak_) peak_ = used_;
            return off;
        }
        return kNone;
    }
    void release(size_t off, size_t bytes) {
        bytes = round_granule(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

// Byte plan of one batch: workspace block [grouped workspace | ASCII |
// records | position offsets | positions] and resident block [ISA | LCP |
// block table].
struct BatchPlan {
    BatchLayout L;
    int np = 0;
    int64_t n = 0, in_bytes = 0, stride = 0;
    int levels = 0;
    size_t o_ascii = 0, o_out = 0, o_off = 0, o_pos = 0, work = 0;
    size_t o_lcp = 0, o_table = 0, resident = 0;
};

BatchPlan plan_batch(const int64_t *lens, int np) {
    BatchPlan P;
    P.np = np;
    int64_t pmax = 1;
    for (int p = 0; p < np; ++p) {
        const int64_t t = lens[2 * p] + lens[2 * p + 1] + 2;
        P.n += t;
        P.in_bytes += lens[2 * p] + lens[2 * p + 1];
        pmax = t > pmax ? t : pmax;
    }
    P.L = batch_layout(P.n);
    size_t off = P.L.total;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    P.o_ascii = take(size_t(P.in_bytes));
    P.o_out = take(sizeof(lor_overlap) * size_t(np));
    P.o_off = take(sizeof(int64_t) * size_t(np + 1));
    P.o_pos = take(sizeof(int32_t) * size_t(P.n));  // positions never exceed n
    P.work = off;
    // whole blocks inside one pair's rank range: at most pmax / 32
    P.levels = bit_width_u64(uint64_t(pmax / kRmqBlock > 0 ? pmax / kRmqBlock : 1));
    P.stride = rmq_row_stride_of(rmqb_blocks(P.n));
    P.o_lcp = align256(sizeof(int32_t) * size_t(P.n));
    P.o_table = P.o_lcp + align256(sizeof(int32_t) * size_t(P.n));
    P.resident = P.o_table + sizeof(int32_t) * size_t(P.levels) * size_t(P.stride);
    return P;
}

struct Resident {
    size_t off = 0, bytes = 0;
    int32_t *isa = nullptr, *lcp = nullptr, *table = nullptr;
    int64_t stride = 0;
    int live = 0;  // requests of the batch not yet released
};

struct Request {
    int64_t id = 0;
    uint64_t tag = 0;
    const uint8_t *a = nullptr, *b = nullptr;
    int64_t la = 0, lb = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = LOR_OK;
    int batch_pairs = 0;
    lor_overlap ov{};
    std::vector<int32_t> pos;
    std::shared_ptr<Resident> res;
    int64_t text_off = 0;  // offset of S1#S2$ inside the batch text
    bool polled = false;
    bool solo = false;  // runs in a batch of its own (its earlier batch failed on an input error)
};

// out[i] = LCP of suffixes P[i], Q[i] of the pair text at [off, off + len) of
// a batch text, from the batch ISA, LCP and block table (host-validated
// queries).
__global__ void k_serve_query(const int32_t *__restrict__ table, int64_t stride, const int32_t *__restrict__ isa,
                              const int32_t *__restrict__ lcp, int64_t off, int64_t len,
                              const int32_t *__restrict__ P,
                              const int32_t *__restrict__ Q, int nq, int32_t *__restrict__ out, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const int32_t p = P[i], q = Q[i];
    if (p < 0 || p >= len || q < 0 || q >= len) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    if (p == q) {
        out[i] = int32_t(len - p);
        return;
    }
    int64_t r1 = isa[off + p], r2 = isa[off + q];
    if (r1 > r2) {
        const int64_t t = r1;
        r1 = r2;
        r2 = t;
    }
    if (r1 == r2) {
        atomicCAS(status, 0, LOR_ERR_BAD_INPUT);
        out[i] = -1;
        return;
    }
    out[i] = rmqb_range_min(table, stride, lcp, r1 + 1, r2);
}

}  // namespace
}  // namespace lor

using namespace lor;

struct lor_server {
    lor_server_config cfg{};
    int device = 0;
    char *base = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_mem, cv_done;
    std::deque<Request *> pending, done;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_id = 1;
    bool stop = false;
    int in_flight = 0;
    lor_server_stats st{};
    std::vector<std::thread> threads;
    std::chrono::steady_clock::time_point t0;
    std::mutex qmu;
    cudaStream_t qs = nullptr;
    int32_t *dq = nullptr, *hq = nullptr;  // 3 * kQueryCap: p, q, answers
    // Device status slots: one per worker, then one for the query stream.  A
    // worker's kernels record errors only in its own slot (set_status_slot),
    // and the worker reads and clears only that slot, so concurrent batches
    // never see or erase each other's errors.
    int *dstatus = nullptr;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Oldest waiting requests that fit in the reservation as one batch of at most
// `limit` pairs; on success they are moved to *batch and their blocks taken.
bool admit(lor_server *S, int limit, std::vector<Request *> *batch, BatchPlan *plan, size_t *off_w,
           size_t *off_r) {
    std::vector<int64_t> lens;
    int np = 0;
    int64_t n = 0;
    if (!S->pending.empty() && S->pending.front()->solo) limit = 1;
    for (Request *r : S->pending) {
        if (np == limit || (np > 0 && r->solo)) break;
        const int64_t add = r->la + r->lb + 2;
        if (np > 0 && n + add > S->cfg.max_batch_symbols) break;
        n += add;
        lens.push_back(r->la);
        lens.push_back(r->lb);
        ++np;
    }
    if (np == 0) return false;
    *plan = plan_batch(lens.data(), np);
    *off_w = S->arena.alloc(plan->work);
    if (*off_w == kNone) return false;
    *off_r = S->arena.alloc(plan->resident);
    if (*off_r == kNone) {
        S->arena.release(*off_w, plan->work);
        return false;
    }
    batch->assign(S->pending.begin(), S->pending.begin() + np);
    S->pending.erase(S->pending.begin(), S->pending.begin() + np);
    return true;
}

int run_batch(lor_server *S, int *d_status, const std::vector<Request *> &batch, const BatchPlan &P, char *wsb,
              const std::shared_ptr<Resident> &res, cudaStream_t s, std::vector<int64_t> *offs,
              std::vector<lor_overlap> *outs, std::vector<int32_t> *hpos) {
    const int np = P.np;
    std::vector<int64_t> lens(2 * size_t(np));
    uint8_t *ascii = (uint8_t *)(wsb + P.o_ascii);
    int64_t in = 0;
    for (int p = 0; p < np; ++p) {
        const Request *r = batch[p];
        lens[2 * p] = r->la;
        lens[2 * p + 1] = r->lb;
        if (r->la) LOR_CUDA_TRY(cudaMemcpyAsync(ascii + in, r->a, size_t(r->la), cudaMemcpyHostToDevice, s));
        in += r->la;
        if (r->lb) LOR_CUDA_TRY(cudaMemcpyAsync(ascii + in, r->b, size_t(r->lb), cudaMemcpyHostToDevice, s));
        in += r->lb;
    }
    lor_overlap *dout = (lor_overlap *)(wsb + P.o_out);
    int64_t *doff = (int64_t *)(wsb + P.o_off);
    int32_t *dpos = (int32_t *)(wsb + P.o_pos);
    const GroupOutputs o{dout, doff, dpos, P.n, 0};
    int64_t found = 0;
    int rc = batch_group(ascii, lens.data(), np, P.n, wsb, P.L.total, P.L, P.n, o, &found, s);
    if (rc) return rc;
    LOR_CUDA_TRY(cudaMemcpyAsync(res->isa, wsb + P.L.isa, sizeof(int32_t) * size_t(P.n),
                                 cudaMemcpyDeviceToDevice, s));
    LOR_CUDA_TRY(cudaMemcpyAsync(res->lcp, wsb + P.L.lcp, sizeof(int32_t) * size_t(P.n),
                                 cudaMemcpyDeviceToDevice, s));
    rc = rmq_block_levels(res->lcp, P.n, P.levels, res->table, s);
    if (rc) return rc;
    outs->resize(np);
    offs->resize(np + 1);
    LOR_CUDA_TRY(cudaMemcpyAsync(outs->data(), dout, sizeof(lor_overlap) * np, cudaMemcpyDeviceToHost, s));
    LOR_CUDA_TRY(cudaMemcpyAsync(offs->data(), doff, sizeof(int64_t) * (np + 1), cudaMemcpyDeviceToHost, s));
    rc = read_status_slot(d_status, s);  // this worker's errors only
    if (rc) return rc;
    const int64_t total = (*offs)[np];
    if (total < 0 || total > P.n) return LOR_ERR_BAD_INPUT;
    hpos->resize(size_t(total));
    if (total) {
        LOR_CUDA_TRY(cudaMemcpyAsync(hpos->data(), dpos, sizeof(int32_t) * size_t(total),
                                     cudaMemcpyDeviceToHost, s));
        LOR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LOR_OK;
}

void worker_main(lor_server *S, int w) {
    cudaSetDevice(S->device);
    int *d_status = S->dstatus + w;
    set_status_slot(d_status);  // every launch of this thread records errors here
    cudaStream_t s = nullptr;
    const bool stream_ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    std::vector<Request *> batch;
    std::vector<int64_t> offs;
    std::vector<lor_overlap> outs;
    std::vector<int32_t> hpos;
    for (;;) {
        BatchPlan P;
        size_t off_w = kNone, off_r = kNone;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            bool counted = false;
            for (;;) {
                if (S->stop) break;
                if (S->pending.empty()) {
                    S->cv_work.wait(lk);
                    continue;
                }
                int limit = S->cfg.max_batch_pairs;
                bool ok = admit(S, limit, &batch, &P, &off_w, &off_r);
                // Nothing else is running: rather than wait, try smaller batches.
                while (!ok && S->in_flight == 0 && limit > 1) {
                    limit = (limit + 1) / 2;
                    ok = admit(S, limit, &batch, &P, &off_w, &off_r);
                }
                if (ok) break;
                if (!counted) {
                    S->st.admission_waits++;
                    counted = true;
                }
                S->cv_mem.wait(lk);
            }
            if (S->stop) break;
            S->in_flight++;
            S->st.batches++;
            S->st.pairs += P.np;
            S->st.bases += P.in_bytes;
        }
        const double ta = S->now();
        for (Request *r : batch) r->t_admit = ta;
        auto res = std::make_shared<Resident>();
        res->off = off_r;
        res->bytes = P.resident;
        res->isa = (int32_t *)(S->base + off_r);
        res->lcp = (int32_t *)(S->base + off_r + P.o_lcp);
        res->table = (int32_t *)(S->base + off_r + P.o_table);
        res->stride = P.stride;
        res->live = P.np;
        int rc = stream_ok ? run_batch(S, d_status, batch, P, S->base + off_w, res, s, &offs, &outs, &hpos)
                           : LOR_ERR_CUDA;
        if (rc == LOR_OK && stream_ok) rc = cudaStreamSynchronize(s) == cudaSuccess ? LOR_OK : LOR_ERR_CUDA;
        if (rc == LOR_ERR_BAD_SYMBOL && P.np > 1) {
            // An input error belongs to one request, not to the batch: run
            // every request of the batch again alone, oldest first, so that
            // only the offending one fails.
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->arena.release(off_w, P.work);
                S->arena.release(off_r, P.resident);
                for (auto it = batch.rbegin(); it != batch.rend(); ++it) {
                    (*it)->solo = true;
                    S->pending.push_front(*it);
                }
                S->st.batches--;
                S->st.pairs -= P.np;
                S->st.bases -= P.in_bytes;
                S->in_flight--;
            }
            batch.clear();
            S->cv_mem.notify_all();
            S->cv_work.notify_all();
            continue;
        }
        const double td = S->now();
        int64_t text_off = 0;
        for (int p = 0; p < P.np; ++p) {
            Request *r = batch[p];
            r->status = rc;
            r->batch_pairs = P.np;
            r->t_done = td;
            r->text_off = text_off;
            text_off += r->la + r->lb + 2;
            if (rc == LOR_OK) {
                r->ov = outs[p];
                const int64_t b0 = offs[p], b1 = offs[p + 1];
                r->pos.assign(hpos.begin() + b0, hpos.begin() + b1);
                r->res = res;
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->arena.release(off_w, P.work);
            if (rc != LOR_OK) S->arena.release(off_r, P.resident);
            for (Request *r : batch) S->done.push_back(r);
            S->st.completed += P.np;
            S->in_flight--;
        }
        batch.clear();
        S->cv_mem.notify_all();
        S->cv_done.notify_all();
    }
    if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" size_t lor_server_batch_bytes(const int64_t *h_lens, int32_t npairs, size_t *h_resident) {
    if (!h_lens || npairs < 1 || npairs > kPairsPerGroup) return 0;
    int64_t n = 0;
    for (int i = 0; i < 2 * npairs; ++i) {
        if (h_lens[i] < 0) return 0;
        n += h_lens[i];
    }
    n += 2 * int64_t(npairs);
    if (n > LOR_MAX_N) return 0;
    const BatchPlan P = plan_batch(h_lens, npairs);
    if (h_resident) *h_resident = P.resident;
    return P.work;
}

extern "C" int lor_server_create(const lor_server_config *cfg, lor_server **out) {
    if (!cfg || !out) return LOR_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->workers < 1 || cfg->workers > kMaxWorkers || cfg->max_batch_pairs < 1 ||
        cfg->max_batch_pairs > kPairsPerGroup || cfg->max_batch_symbols < 1 ||
        cfg->max_batch_symbols > kGroupSymbolCap || cfg->hbm_budget_bytes < kGranule)
        return LOR_ERR_INVALID_ARG;
    auto S = std::make_unique<lor_server>();
    S->cfg = *cfg;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) return LOR_ERR_CUDA;
    const size_t budget = cfg->hbm_budget_bytes & ~(kGranule - 1);
    if (cudaMalloc(&S->base, budget) != cudaSuccess) {
        cudaGetLastError();
        return LOR_ERR_CUDA;
    }
    S->arena.init(budget);
    int lo = 0, hi = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&S->qs, cudaStreamNonBlocking, hi) == cudaSuccess &&
              cudaMalloc(&S->dq, sizeof(int32_t) * 3 * kQueryCap) == cudaSuccess &&
              cudaHostAlloc(&S->hq, sizeof(int32_t) * 3 * kQueryCap, cudaHostAllocDefault) == cudaSuccess &&
              cudaMalloc(&S->dstatus, sizeof(int) * (kMaxWorkers + 1)) == cudaSuccess &&
              cudaMemset(S->dstatus, 0, sizeof(int) * (kMaxWorkers + 1)) == cudaSuccess;
    if (!ok) {
        if (S->qs) cudaStreamDestroy(S->qs);
        if (S->dstatus) cudaFree(S->dstatus);
        if (S->dq) cudaFree(S->dq);
        if (S->hq) cudaFreeHost(S->hq);
        cudaFree(S->base);
        return LOR_ERR_CUDA;
    }
    lor_server *srv = S.release();
    for (int w = 0; w < cfg->workers; ++w) srv->threads.emplace_back(worker_main, srv, w);
    *out = srv;
    return LOR_OK;
}

extern "C" int lor_server_submit(lor_server *S, const uint8_t *h_a, int64_t len_a, const uint8_t *h_b,
                                 int64_t len_b, uint64_t tag, int64_t *out_id) {
    if (!S || !out_id || len_a < 0 || len_b < 0 || (len_a && !h_a) || (len_b && !h_b))
        return LOR_ERR_INVALID_ARG;
    if (len_a + len_b + 2 > LOR_MAX_N) return LOR_ERR_TOO_LARGE;
    const int64_t lens[2] = {len_a, len_b};
    const BatchPlan P = plan_batch(lens, 1);
    if (round_granule(P.work) + round_granule(P.resident) > S->arena.size()) return LOR_ERR_TOO_LARGE;
    auto r = std::make_unique<Request>();
    r->tag = tag;
    r->a = h_a;
    r->b = h_b;
    r->la = len_a;
    r->lb = len_b;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return LOR_ERR_CANCELLED;
        r->id = S->next_id++;
        r->t_submit = S->now();
        *out_id = r->id;
        S->pending.push_back(r.get());
        S->reqs.emplace(r->id, std::move(r));
        S->st.submitted++;
    }
    S->cv_work.notify_one();
    return LOR_OK;
}

extern "C" int lor_server_poll(lor_server *S, lor_served *out, int32_t cap, int32_t timeout_ms) {
    if (!S || !out || cap < 1) return LOR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && timeout_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !S->done.empty(); });
    int k = 0;
    while (k < cap && !S->done.empty()) {
        Request *r = S->done.front();
        S->done.pop_front();
        r->polled = true;
        lor_served &o = out[k++];
        o.id = r->id;
        o.tag = r->tag;
        o.status = r->status;
        o.batch_pairs = r->batch_pairs;
        o.ov = r->ov;
        o.positions = r->pos.empty() ? nullptr : r->pos.data();
        o.t_submit = r->t_submit;
        o.t_admit = r->t_admit;
        o.t_done = r->t_done;
    }
    return k;
}

extern "C" int lor_server_query(lor_server *S, int64_t id, const int32_t *h_p, const int32_t *h_q, int32_t nq,
                                int32_t *h_out) {
    if (!S || nq < 0) return LOR_ERR_INVALID_ARG;
    if (nq == 0) return LOR_OK;
    if (!h_p || !h_q || !h_out) return LOR_ERR_INVALID_ARG;
    std::shared_ptr<Resident> res;
    int64_t off = 0, len = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second->polled || !it->second->res) return LOR_ERR_INVALID_ARG;
        res = it->second->res;
        off = it->second->text_off;
        len = it->second->la + it->second->lb + 2;
    }
    for (int32_t i = 0; i < nq; ++i)
        if (h_p[i] < 0 || h_p[i] >= len || h_q[i] < 0 || h_q[i] >= len) return LOR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> qk(S->qmu);
    cudaSetDevice(S->device);
    int *status = S->dstatus + kMaxWorkers;  // the query stream's own slot
    for (int32_t b = 0; b < nq; b += kQueryCap) {
        const int c = nq - b < kQueryCap ? nq - b : kQueryCap;
        memcpy(S->hq, h_p + b, sizeof(int32_t) * c);
        memcpy(S->hq + kQueryCap, h_q + b, sizeof(int32_t) * c);
        LOR_CUDA_TRY(cudaMemcpyAsync(S->dq, S->hq, sizeof(int32_t) * 2 * kQueryCap, cudaMemcpyHostToDevice, S->qs));
        k_serve_query<<<unsigned(cdiv(c, 128)), 128, 0, S->qs>>>(res->table, res->stride, res->isa, res->lcp, off, len, S->dq,
                                                                 S->dq + kQueryCap, c, S->dq + 2 * kQueryCap,
                                                                 status);
        LOR_LAUNCH_CHECK();
        LOR_CUDA_TRY(cudaMemcpyAsync(S->hq + 2 * kQueryCap, S->dq + 2 * kQueryCap, sizeof(int32_t) * c,
                                     cudaMemcpyDeviceToHost, S->qs));
        LOR_CUDA_TRY(cudaStreamSynchronize(S->qs));
        memcpy(h_out + b, S->hq + 2 * kQueryCap, sizeof(int32_t) * c);
    }
    const int qrc = read_status_slot(status, S->qs);
    if (qrc != LOR_OK) return qrc;
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.queries += nq;
    return LOR_OK;
}

extern "C" int lor_server_release(lor_server *S, int64_t id) {
    if (!S) return LOR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second->polled) return LOR_ERR_INVALID_ARG;
        std::shared_ptr<Resident> res = it->second->res;
        S->reqs.erase(it);
        S->st.released++;
        if (!res || --res->live > 0) return LOR_OK;
        S->arena.release(res->off, res->bytes);
    }
    S->cv_mem.notify_all();
    return LOR_OK;
}

extern "C" int lor_server_stats_get(lor_server *S, lor_server_stats *out) {
    if (!S || !out) return LOR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->reserved_bytes = S->arena.size();
    out->in_use_bytes = S->arena.used();
    out->peak_bytes = S->arena.peak();
    out->pending = int32_t(S->pending.size());
    out->in_flight = S->in_flight;
    return LOR_OK;
}

extern "C" double lor_server_now(lor_server *S) { return S ? S->now() : 0.0; }

extern "C" int lor_server_destroy(lor_server *S) {
    if (!S) return LOR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_mem.notify_all();
    for (auto &t : S->threads) t.join();
    cudaSetDevice(S->device);
    cudaStreamSynchronize(S->qs);
    cudaStreamDestroy(S->qs);
    cudaFree(S->dq);
    cudaFree(S->dstatus);
    cudaFreeHost(S->hq);
    cudaFree(S->base);
    delete S;
    return LOR_OK;
}
