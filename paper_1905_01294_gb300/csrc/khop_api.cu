// C ABI entry points of the counting calls: argument checks, per-graph call
// ordering, and dispatch to the plain or the bit-sliced batched path.
#include <algorithm>
#include <vector>

#include "khop_internal.cuh"

using namespace khop;

namespace {

// The single query (seed, k) of a neighbourhood call, in device memory.
__global__ void one_query_kernel(uint32_t *q, uint32_t seed, uint32_t k) {
    q[0] = seed;
    q[1] = k;
}

// The seed is in its own neighbourhood (also when the query needed no traversal).
__global__ void seed_bit_kernel(uint32_t *bits, uint32_t seed) {
    atomicOr(&bits[seed >> 5], 1u << (seed & 31));
}

// Vertex list from a bitmap, ascending: every block takes a contiguous run of
// words; cnt[b] = bits in block b's run.
__global__ void count_bits_kernel(const uint32_t *bits, uint64_t nw, uint64_t per_block, uint32_t *cnt) {
    __shared__ unsigned s[32];
    const uint64_t w0 = (uint64_t)blockIdx.x * per_block, w1 = min(w0 + per_block, nw);
    unsigned c = 0;
    for (uint64_t i = w0 + threadIdx.x; i < w1; i += blockDim.x) c += (unsigned)__popc(bits[i]);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (unsigned i = 0; i < blockDim.x / 32; ++i) t += s[i];
        cnt[blockIdx.x] = t;
    }
}

// Writes the ids of block b's run at offset sum(cnt[0..b)); ids beyond
// `capacity` are dropped; block 0 writes the total to *size.  One thread per
// word, words in order.
__global__ void write_ids_kernel(const uint32_t *bits, uint64_t nw, uint64_t per_block, const uint32_t *cnt,
                                 uint32_t *ids, uint64_t capacity, uint64_t *size) {
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_warp[32];
    if (threadIdx.x == 0) {
        unsigned long long b = 0, t = 0;
        for (unsigned i = 0; i < gridDim.x; ++i) {
            if (i < blockIdx.x) b += cnt[i];
            t += cnt[i];
        }
        s_base = b;
        if (blockIdx.x == 0) *size = t;
    }
    __syncthreads();
    const uint64_t w0 = (uint64_t)blockIdx.x * per_block, w1 = min(w0 + per_block, nw);
    unsigned long long base = s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t c0 = w0; c0 < w1; c0 += blockDim.x) {
        const uint64_t i = c0 + threadIdx.x;
        const uint32_t x = i < w1 ? bits[i] : 0u;
        const unsigned c = (unsigned)__popc(x);
        const unsigned incl = warp_inclusive_sum(c);
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        unsigned before = incl - c, total = 0;
        for (unsigned j = 0; j < blockDim.x / 32; ++j) {
            if (j < (unsigned)warp) before += s_warp[j];
            total += s_warp[j];
        }
        unsigned long long o = base + before;
        for (uint32_t y = x; y; y &= y - 1, ++o)
            if (o < capacity) ids[o] = (uint32_t)((i << 5) + (uint64_t)__ffs(y) - 1);
        base += total;
        __syncthreads();
    }
}

// Runs the single query (seed, k) with every round on the grid path; the
// neighbourhood is then plain.V (plus the seed bit); levels, if given, get
// the hop distance of every vertex the rounds discover.
int run_one(khop_graph *g, uint32_t seed, uint32_t k, cudaStream_t st, int32_t *levels = nullptr) {
    uint32_t *q = g->plain.ctl->one_q;
    one_query_kernel<<<1, 1, 0, st>>>(q, seed, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    int rc = plain_launch(g, q, q + 1, 0, 1, (uint64_t *)&g->plain.ctl->one_out, nullptr, nullptr, nullptr, 0,
                          st, true, levels);
    if (rc != KHOP_OK) return rc;
    seed_bit_kernel<<<1, 1, 0, st>>>(g->plain.V, seed);
    return cuda_status(cudaGetLastError());
}

__global__ void seed_level_kernel(int32_t *levels, uint32_t seed) { levels[seed] = 0; }

// BFS parents over the (MIN, SECOND) semiring: parent(v) = the smallest
// in-neighbour u of v with level(u) = level(v) - 1 (v reached, v != s);
// parent(s) = s; unreached vertices get UINT32_MAX.  A warp takes 32
// consecutive vertices (one coalesced read of their levels), then scans the
// in-lists of the reached ones together, one vertex at a time.
template <typename E>
__global__ void parents_kernel(const E *cp, const uint32_t *ri, const int32_t *levels, uint64_t n,
                               uint32_t *parents) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = warp << 5; base < n; base += nwarps << 5) {
        const uint64_t v = base + (uint64_t)lane;
        const int32_t lv = v < n ? levels[v] : -1;
        uint32_t mine = lv == 0 ? (uint32_t)v : 0xffffffffu;
        unsigned todo = __ballot_sync(FULL, lv > 0);
        while (todo) {
            const int L = __ffs(todo) - 1;
            todo &= todo - 1u;
            const uint64_t x = base + (uint64_t)L;
            const int32_t want = __shfl_sync(FULL, lv, L) - 1;
            uint32_t best = 0xffffffffu;
            for (E i = cp[x] + lane; i < cp[x + 1]; i += 32) {
                const uint32_t u = ri[i];
                if (levels[u] == want) best = min(best, u);
            }
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL, best, o));
            if (lane == L) mine = best;
        }
        if (v < n) parents[v] = mine;
    }
}

}  // namespace

extern "C" {

int khop_neighbourhood(khop_graph *g, uint32_t seed, uint32_t k, uint32_t *out_bits, uint64_t *out_count,
                       void *stream) {
    if (!g || !out_bits || seed >= g->n) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK) rc = run_one(g, seed, k, st);
    if (rc == KHOP_OK)
        rc = cuda_status(cudaMemcpyAsync(out_bits, g->plain.V, (uint64_t)g->nw * 4, cudaMemcpyDeviceToDevice, st));
    if (rc == KHOP_OK && out_count)
        rc = cuda_status(cudaMemcpyAsync(out_count, &g->plain.ctl->one_out, 8, cudaMemcpyDeviceToDevice, st));
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

int khop_levels(khop_graph *g, uint32_t seed, uint32_t k, int32_t *out_levels, uint32_t *out_parents,
                void *stream) {
    if (!g || !out_levels || seed >= g->n) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK) rc = cuda_status(cudaMemsetAsync(out_levels, 0xff, g->n * sizeof(int32_t), st));
    if (rc == KHOP_OK) rc = run_one(g, seed, k, st, out_levels);
    if (rc == KHOP_OK) {
        seed_level_kernel<<<1, 1, 0, st>>>(out_levels, seed);
        rc = cuda_status(cudaGetLastError());
    }
    if (rc == KHOP_OK && out_parents) {
        const int blocks = g->num_sms * 8;
        if (g->ewidth == 4)
            parents_kernel<uint32_t><<<blocks, 256, 0, st>>>((const uint32_t *)g->cp, g->ri, out_levels, g->n,
                                                            out_parents);
        else
            parents_kernel<unsigned long long><<<blocks, 256, 0, st>>>((const unsigned long long *)g->cp, g->ri,
                                                                      out_levels, g->n, out_parents);
        rc = cuda_status(cudaGetLastError());
    }
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

int khop_neighbourhood_list(khop_graph *g, uint32_t seed, uint32_t k, uint32_t *out_ids, uint64_t capacity,
                            uint64_t *out_size, void *stream) {
    if (!g || !out_size || (capacity && !out_ids) || seed >= g->n) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK) rc = run_one(g, seed, k, st);
    if (rc == KHOP_OK) {
        // the frontier bitmaps are free after the launch (the next one zeroes them)
        const uint64_t nw = g->nw;
        const uint64_t blocks = std::min<uint64_t>((uint64_t)g->num_sms * 4, nw);
        const uint64_t per_block = (nw + blocks - 1) / blocks;
        const uint64_t used = (nw + per_block - 1) / per_block;
        uint32_t *cnt = g->plain.F[0];
        count_bits_kernel<<<(unsigned)used, 256, 0, st>>>(g->plain.V, nw, per_block, cnt);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) {
            write_ids_kernel<<<(unsigned)used, 256, 0, st>>>(g->plain.V, nw, per_block, cnt, out_ids, capacity,
                                                              out_size);
            e = cudaGetLastError();
        }
        rc = cuda_status(e);
    }
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

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
    if (mode < KHOP_MODE_AUTO || mode > KHOP_MODE_BATCHED256) return KHOP_EINVAL;
    if (nseeds == 0) return KHOP_OK;
    if (!seeds || !ks || !out_counts) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool batched = mode == KHOP_MODE_BATCHED64 || mode == KHOP_MODE_BATCHED128 ||
                         mode == KHOP_MODE_BATCHED256 || (mode == KHOP_MODE_AUTO && nseeds >= 2);
    const int lw = mode == KHOP_MODE_BATCHED256 ? 4 : (mode == KHOP_MODE_BATCHED128 ? 2 : 1);
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    if (rc == KHOP_OK) {
        if (batched) {
            rc = ensure_batch_state(g, lw);
            if (rc == KHOP_OK) rc = batch_launch(g, seeds, ks, nseeds, out_counts, st, lw);
            g->last_lw = lw;
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
    const BatchState &bs = g->last_lw == 4 ? g->batch4 : (g->last_lw == 2 ? g->batch2 : g->batch);
    if (bs.ctl) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(v, bs.ctl->pad, sizeof(v), cudaMemcpyDeviceToHost);
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
