// C ABI entry points of the counting calls: argument checks, per-graph call
// ordering, and dispatch to the plain or the bit-sliced batched path.
#include <algorithm>
#include <vector>

#include "khop_internal.cuh"

using namespace khop;

extern "C" {

int khop_count_ex(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nseeds,
                  uint64_t *out_counts, uint64_t *out_te, khop_query_stats *out_stats,
                  uint64_t *per_hop, uint32_t hop_stride, void *stream) {
    if (!g) return KHOP_EINVAL;
    if (nseeds == 0) return KHOP_OK;
    if (!seeds || !ks || !out_counts) return KHOP_EINVAL;
    if (per_hop && hop_stride == 0) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK)
        rc = plain_launch(g, seeds, ks, 0, nseeds, out_counts, out_te, out_stats, per_hop,
                          hop_stride, st);
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

int khop_count(khop_graph *g, const uint32_t *seeds, uint64_t nseeds, uint32_t k,
               uint64_t *out_counts, void *stream) {
    if (!g) return KHOP_EINVAL;
    if (nseeds == 0) return KHOP_OK;
    if (!seeds || !out_counts) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK)
        rc = plain_launch(g, seeds, nullptr, k, nseeds, out_counts, nullptr, nullptr, nullptr, 0, st);
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

int khop_count_mixed(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nseeds,
                     uint64_t *out_counts, int mode, void *stream) {
    if (!g) return KHOP_EINVAL;
    if (mode < KHOP_MODE_AUTO || mode > KHOP_MODE_BATCHED64) return KHOP_EINVAL;
    if (nseeds == 0) return KHOP_OK;
    if (!seeds || !ks || !out_counts) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool batched = mode == KHOP_MODE_BATCHED64 || (mode == KHOP_MODE_AUTO && nseeds >= 2);
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK) {
        if (batched) {
            rc = ensure_batch_state(g);
            if (rc == KHOP_OK) rc = batch_launch(g, seeds, ks, nseeds, out_counts, st);
        } else {
            rc = plain_launch(g, seeds, ks, 0, nseeds, out_counts, nullptr, nullptr, nullptr, 0, st);
        }
    }
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

int khop_batch_stats(khop_graph *g, uint64_t *batches, uint64_t *bytes, uint64_t *rounds,
                     uint64_t *pull_rounds) {
    if (!g) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    unsigned long long v[4] = {0, 0, 0, 0};
    if (g->batch.ctl) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(v, g->batch.ctl->pad, sizeof(v), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (batches) *batches = v[0];
    if (bytes) *bytes = v[1];
    if (rounds) *rounds = v[2];
    if (pull_rounds) *pull_rounds = v[3];
    return KHOP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: coordinate descent over the tunables, each candidate timed with
// CUDA events (best of three runs) on the caller's seeds; counts never depend
// on the tuning, so only the time decides.

namespace {

float time_plain(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int *rc) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, st);
        *rc = plain_launch(g, seeds, ks, 0, nq, out, nullptr, nullptr, nullptr, 0, st);
        cudaEventRecord(b, st);
        if (*rc != KHOP_OK || cudaEventSynchronize(b) != cudaSuccess) return 1e30f;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    return best;
}

float time_batch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int *rc) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, st);
        *rc = batch_launch(g, seeds, ks, nq, out, st);
        cudaEventRecord(b, st);
        if (*rc != KHOP_OK || cudaEventSynchronize(b) != cudaSuccess) return 1e30f;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    return best;
}

}  // namespace

extern "C" int khop_autotune(khop_graph *g, const uint32_t *seeds, const uint32_t *ks_in,
                             uint64_t nq, uint32_t k, void *stream, khop_tuning *chosen) {
    if (!g || !seeds || nq == 0 || (!ks_in && k == 0)) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc != KHOP_OK) return rc;
    rc = ensure_batch_state(g);
    if (rc != KHOP_OK) return rc;
    uint64_t *out = nullptr;
    uint32_t *ks = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&out, nq * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&ks, nq * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        if (ks_in) {
            e = cudaMemcpyAsync(ks, ks_in, nq * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
        } else {
            std::vector<uint32_t> hk(nq, k);
            e = cudaMemcpyAsync(ks, hk.data(), nq * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        cudaFree(out);
        cudaFree(ks);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        return cuda_status(e);
    }
    khop_tuning& t = g->tune;
    const int dir0 = t.direction;
    t.direction = KHOP_DIR_AUTO;
    // plain path: grid shape, push tile, alpha, beta
    struct Shape { int block, per_sm; };
    const Shape shapes[] = {{512, 2}, {1024, 1}, {256, 4}, {512, 1}};
    float best = time_plain(g, seeds, ks, nq, out, st, a, b, &rc);
    Shape bs{t.block_threads, t.blocks_per_sm};
    for (const Shape &s : shapes) {
        t.block_threads = s.block;
        t.blocks_per_sm = s.per_sm;
        const float ms = time_plain(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < best) { best = ms; bs = s; }
    }
    t.block_threads = bs.block;
    t.blocks_per_sm = bs.per_sm;
    int best_tile = t.push_tile;
    for (int tile : {512, 1024, 2048, 4096}) {
        t.push_tile = tile;
        const float ms = time_plain(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < best) { best = ms; best_tile = tile; }
    }
    t.push_tile = best_tile;
    float best_alpha = t.alpha;
    for (float al : {4.0f, 8.0f, 14.0f, 24.0f, 40.0f}) {
        t.alpha = al;
        const float ms = time_plain(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < best) { best = ms; best_alpha = al; }
    }
    t.alpha = best_alpha;
    float best_beta = t.beta;
    for (float be : {8.0f, 24.0f, 64.0f}) {
        t.beta = be;
        const float ms = time_plain(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < best) { best = ms; best_beta = be; }
    }
    t.beta = best_beta;
    // batched path: alpha, beta
    float bbest = time_batch(g, seeds, ks, nq, out, st, a, b, &rc);
    float bal = t.batch_alpha;
    for (float al : {2.0f, 5.0f, 14.0f, 30.0f, 60.0f}) {
        t.batch_alpha = al;
        const float ms = time_batch(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < bbest) { bbest = ms; bal = al; }
    }
    t.batch_alpha = bal;
    float bbe = t.batch_beta;
    for (float be : {6.0f, 24.0f, 100.0f}) {
        t.batch_beta = be;
        const float ms = time_batch(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < bbest) { bbest = ms; bbe = be; }
    }
    t.batch_beta = bbe;
    int btile = t.batch_push_tile;
    for (int tile : {1024, 2048, 4096}) {
        t.batch_push_tile = tile;
        const float ms = time_batch(g, seeds, ks, nq, out, st, a, b, &rc);
        if (ms < bbest) { bbest = ms; btile = tile; }
    }
    t.batch_push_tile = btile;
    t.direction = dir0;
    e = cudaStreamSynchronize(st);
    cudaFree(out);
    cudaFree(ks);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc == KHOP_OK) rc = cuda_status(e);
    if (rc == KHOP_OK) rc = mark_done(g, st);
    if (chosen) *chosen = t;
    return rc;
}
