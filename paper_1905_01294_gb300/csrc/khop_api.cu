// C ABI entry points of the counting calls: argument checks, per-graph call
// ordering, and dispatch to the plain or the bit-sliced batched path.
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
