// tune.cu -- the autotuner of the batched pipeline's launch parameters.
//
// Coordinate descent over the parameters of lor_tune, timed on the caller's
// own batch: for each parameter in turn every candidate value is tried with
// the others held at the best found so far, and a value is kept only when it
// makes lor_batch_overlap faster.  The candidates are few (at most four per
// parameter), so a tuning run costs a dozen or so timed batches.
#include <vector>

#include "common.cuh"


namespace {

int time_batch(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs, lor_overlap *d_out,
               int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes, int reps,
               cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *ms) {
    int rc = lor_batch_overlap(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes,
                               (lor_stream_t)s);
    if (rc) return rc;
    if (cudaEventRecord(e0, s) != cudaSuccess) return LOR_ERR_CUDA;
    for (int r = 0; r < reps; ++r) {
        rc = lor_batch_overlap(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes,
                               (lor_stream_t)s);
        if (rc) return rc;
    }
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return LOR_ERR_CUDA;
    float t = 0;
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return LOR_ERR_CUDA;
    *ms = double(t) / reps;
    return lor_device_status((lor_stream_t)s);
}

}  // namespace

extern "C" int lor_autotune_batch(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs,
                                  lor_overlap *d_out, int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap,
                                  void *d_ws, size_t ws_bytes, int32_t reps, lor_stream_t stream, lor_tune *best,
                                  double *best_ms) {
    if (!best || !best_ms || reps < 1 || reps > 100) return LOR_ERR_INVALID_ARG;
    lor_tune cur;
    lor_tune_get(&cur);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return LOR_ERR_CUDA;
    }
    double cur_ms = 0;
    int rc = time_batch(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes, reps, s, e0,
                        e1, &cur_ms);
    // (parameter, candidate values) in the order they are tuned
    struct Knob {
        int32_t lor_tune::*field;
        std::vector<int32_t> values;
    };
    const Knob knobs[] = {
        {&lor_tune::level0_key_bits, {30, 40, 48, 56}},
        {&lor_tune::digit_bits, {6, 7, 8}},
        {&lor_tune::sort_items_64, {8, 12, 16}},
        {&lor_tune::sort_items_32, {12, 16}},
        {&lor_tune::merge_items, {2, 4, 8}},
    };
    for (const Knob &k : knobs) {
        for (int32_t v : k.values) {
            if (rc) break;
            if (cur.*k.field == v) continue;
            lor_tune cand = cur;
            cand.*k.field = v;
            rc = lor_tune_set(&cand);
            if (rc) break;
            double ms = 0;
            rc = time_batch(d_ascii, h_lens, npairs, d_out, d_pos_off, d_pos, pos_cap, d_ws, ws_bytes, reps, s,
                            e0, e1, &ms);
            if (rc) break;
            if (ms < cur_ms) {
                cur = cand;
                cur_ms = ms;
            }
        }
    }
    lor_tune_set(&cur);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = cur;
    *best_ms = cur_ms;
    return rc;
}
