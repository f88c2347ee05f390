// Continuous-batching request server for the k-hop count (khop_server_*).
//
// Requests (graph, seed, k) arrive from any host thread.  A worker thread
// keeps them in per-graph FIFO queues by k and runs them in cohorts of up to
// 64 on bit-sliced batch slots: whenever a slot is free, the oldest waiting
// request's k picks the cohort, which is filled first with requests of that
// k and then with requests of smaller k (they finish earlier within the same
// sweeps), oldest first.  Slots are allocated on demand, each only if free
// device memory (minus a margin) and the server's budget admit it, up to
// max_batches per graph; while every slot is busy, requests wait.  Each slot
// has its own stream and its cohort kernel uses a part of the SMs, so the
// cohorts of several slots run side by side on the device while the worker
// admits and completes others.  This is the GPU counterpart of the paper's
// design that serves many concurrent queries from a thread pool (Sec. II).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>
#include <time.h>

#include "khop_internal.cuh"

namespace {

using namespace khop;

constexpr int kLaneWords = 64 * 3 + 2;   // seeds, ks, order, then the batch count (u64)
constexpr uint64_t kMarginBytes = 1ull << 30;

uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Request {
    uint64_t ticket;
    khop_graph *g;
    uint32_t seed, k;
    uint64_t t_submit;
};

constexpr size_t kPlainCohort = 2;   // cohorts this small run on the plain kernel

struct Slot {
    BatchState st;
    PlainState pst;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *d_lanes = nullptr;
    uint64_t *d_out = nullptr;
    uint32_t *h_lanes = nullptr;   // pinned
    uint64_t *h_out = nullptr;     // pinned
    std::vector<Request> reqs;     // the cohort in flight
    bool busy = false;
    bool timed_out = false;
    uint64_t t_launch = 0;
};

struct GraphCtx {
    khop_graph *g = nullptr;
    std::deque<Request> pending[64];   // by min(k, 63)
    uint64_t npending = 0;
    std::vector<Slot *> slots;
};

}  // namespace

struct khop_server {
    khop_server_opts opts{};
    int device = 0;
    int grid_ctas = 0;
    std::mutex mu;
    std::condition_variable cv_in, cv_out;
    std::deque<Request> inbox;
    std::deque<khop_result> outbox;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, steps = 0, slots_allocated = 0;
    uint64_t queued = 0;            // submitted and not yet completed
    uint64_t mem_used = 0;          // device bytes of the slots
    std::map<khop_graph *, GraphCtx *> graphs;   // worker-owned
    std::thread worker;
};

namespace {

void post(khop_server *s, const Request &r, uint64_t count, int status) {
    khop_result res{};
    res.ticket = r.ticket;
    res.count = count;
    res.status = status;
    res.k = r.k;
    res.t_submit_ns = r.t_submit;
    res.t_done_ns = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    s->outbox.push_back(res);
    s->completed++;
    s->queued--;
    s->cv_out.notify_all();
}

void free_slot(khop_server *s, Slot *sl) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    free_batch_state(sl->st);
    free_plain_state(sl->pst);
    cudaFree(sl->d_lanes);
    cudaFree(sl->d_out);
    cudaFreeHost(sl->h_lanes);
    cudaFreeHost(sl->h_out);
    if (sl->done) cudaEventDestroy(sl->done);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
    (void)s;
}

// A new slot for ctx if memory and the budget admit it, else null.
Slot *try_alloc_slot(khop_server *s, GraphCtx *ctx) {
    const uint64_t cap = s->opts.max_batches ? s->opts.max_batches : 8;
    if (ctx->slots.size() >= cap) return nullptr;
    const uint64_t need = batch_state_bytes(ctx->g) + plain_state_bytes(ctx->g) + 4096;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return nullptr;
    if ((uint64_t)fr < need + kMarginBytes) return nullptr;
    if (s->opts.mem_budget_bytes && s->mem_used + need > s->opts.mem_budget_bytes) return nullptr;
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) return nullptr;
    uint64_t bytes = 0;
    bool ok;
    {
        // the slot belongs to the server, not to the graph's own accounting
        std::lock_guard<std::mutex> glk(ctx->g->mu);
        ok = alloc_batch_state(ctx->g, sl->st, &bytes) == KHOP_OK;
        if (ok) ctx->g->device_bytes -= bytes;
        ok = ok && alloc_plain_state(ctx->g, sl->pst) == KHOP_OK;
        if (ok) {
            ctx->g->device_bytes -= sl->pst.bytes;
            bytes += sl->pst.bytes;
        }
    }
    ok = ok && cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&sl->d_lanes, kLaneWords * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&sl->d_out, 64 * sizeof(uint64_t)) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl->h_lanes, kLaneWords * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl->h_out, 64 * sizeof(uint64_t)) == cudaSuccess;
    if (!ok) {
        free_slot(s, sl);
        return nullptr;
    }
    s->mem_used += bytes + kLaneWords * 4 + 64 * 8;
    ctx->slots.push_back(sl);
    std::lock_guard<std::mutex> lk(s->mu);
    s->slots_allocated++;
    return sl;
}

// Take the next cohort of ctx: the oldest request's k, then smaller k.
void take_cohort(GraphCtx *ctx, std::vector<Request> &out) {
    int kb = -1;
    uint64_t oldest = ~0ull;
    for (int b = 1; b < 64; ++b)
        if (!ctx->pending[b].empty() && ctx->pending[b].front().t_submit < oldest) {
            oldest = ctx->pending[b].front().t_submit;
            kb = b;
        }
    out.clear();
    for (int b = kb; b >= 1 && out.size() < 64; --b) {
        auto &q = ctx->pending[b];
        while (!q.empty() && out.size() < 64) {
            out.push_back(q.front());
            q.pop_front();
        }
    }
    ctx->npending -= out.size();
}

int launch_cohort(khop_server *s, GraphCtx *ctx, Slot *sl) {
    take_cohort(ctx, sl->reqs);
    const size_t c = sl->reqs.size();
    for (int l = 0; l < 64; ++l) {
        const bool on = (size_t)l < c;
        sl->h_lanes[l] = on ? sl->reqs[l].seed : 0u;
        sl->h_lanes[64 + l] = on ? sl->reqs[l].k : 0u;
        sl->h_lanes[128 + l] = on ? (uint32_t)l : 0xffffffffu;
    }
    const unsigned long long one = 1ull;
    memcpy(sl->h_lanes + 192, &one, sizeof(one));
    cudaError_t e = cudaMemcpyAsync(sl->d_lanes, sl->h_lanes, kLaneWords * sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, sl->stream);
    int rc = cuda_status(e);
    if (rc == KHOP_OK) {
        if (c <= kPlainCohort)   // one or two queries: the single-query kernel is cheaper
            rc = plain_launch_state(ctx->g, sl->pst, sl->d_lanes, sl->d_lanes + 64, c, sl->d_out,
                                    s->grid_ctas, sl->stream);
        else
            rc = batch_launch_slot(ctx->g, sl->st, sl->d_lanes, sl->d_out, s->grid_ctas, sl->stream);
    }
    if (rc == KHOP_OK)
        rc = cuda_status(cudaMemcpyAsync(sl->h_out, sl->d_out, 64 * sizeof(uint64_t),
                                         cudaMemcpyDeviceToHost, sl->stream));
    if (rc == KHOP_OK) rc = cuda_status(cudaEventRecord(sl->done, sl->stream));
    if (rc != KHOP_OK) {
        for (auto &r : sl->reqs) post(s, r, ~0ull, rc);
        sl->reqs.clear();
        return rc;
    }
    sl->busy = true;
    sl->timed_out = false;
    sl->t_launch = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    s->steps++;
    return KHOP_OK;
}

void finish_slot(khop_server *s, Slot *sl, int status) {
    if (!sl->timed_out)
        for (size_t i = 0; i < sl->reqs.size(); ++i)
            post(s, sl->reqs[i], status == KHOP_OK ? sl->h_out[i] : ~0ull, status);
    sl->reqs.clear();
    sl->busy = false;
    sl->timed_out = false;
}

void worker_main(khop_server *s) {
    cudaSetDevice(s->device);
    const uint64_t timeout_ns =
        (uint64_t)(s->opts.wait_timeout_us > 0 ? s->opts.wait_timeout_us : 2000000) * 1000ull;
    std::vector<Request> incoming;
    for (;;) {
        bool stopping;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            stopping = s->stop;
            incoming.assign(s->inbox.begin(), s->inbox.end());
            s->inbox.clear();
        }
        for (const Request &r : incoming) {
            GraphCtx *&ctx = s->graphs[r.g];
            if (!ctx) {
                ctx = new GraphCtx();
                ctx->g = r.g;
            }
            ctx->pending[std::min<uint32_t>(r.k, 63)].push_back(r);
            ctx->npending++;
        }
        incoming.clear();
        // completions
        bool busy = false;
        for (auto &kv : s->graphs)
            for (Slot *sl : kv.second->slots) {
                if (!sl->busy) continue;
                const cudaError_t q = cudaEventQuery(sl->done);
                if (q == cudaSuccess) {
                    finish_slot(s, sl, KHOP_OK);
                } else if (q == cudaErrorNotReady) {
                    busy = true;
                    if (!sl->timed_out && now_ns() - sl->t_launch > timeout_ns) {
                        for (auto &r : sl->reqs) post(s, r, ~0ull, KHOP_ETIMEDOUT);
                        sl->timed_out = true;   // the slot stays reserved until it completes
                    }
                } else {
                    finish_slot(s, sl, KHOP_ECUDA);
                }
            }
        if (stopping) {
            if (busy) {
                for (auto &kv : s->graphs)
                    for (Slot *sl : kv.second->slots)
                        if (sl->busy) {
                            const cudaError_t e = cudaStreamSynchronize(sl->stream);
                            finish_slot(s, sl, e == cudaSuccess ? KHOP_OK : KHOP_ECUDA);
                        }
            }
            for (auto &kv : s->graphs) {
                GraphCtx *ctx = kv.second;
                for (int b = 0; b < 64; ++b)
                    for (auto &r : ctx->pending[b]) post(s, r, ~0ull, KHOP_ESHUTDOWN);
                for (Slot *sl : ctx->slots) free_slot(s, sl);
                delete ctx;
            }
            s->graphs.clear();
            return;
        }
        // admissions: fill every free (or newly admitted) slot
        bool launched = false, pending = false;
        for (auto &kv : s->graphs) {
            GraphCtx *ctx = kv.second;
            while (ctx->npending) {
                Slot *free_sl = nullptr;
                for (Slot *sl : ctx->slots)
                    if (!sl->busy) { free_sl = sl; break; }
                if (!free_sl) free_sl = try_alloc_slot(s, ctx);
                if (!free_sl) {
                    if (ctx->slots.empty()) {
                        // no slot could ever run these: fail them
                        for (int b = 0; b < 64; ++b) {
                            for (auto &r : ctx->pending[b]) post(s, r, ~0ull, KHOP_ENOMEM);
                            ctx->pending[b].clear();
                        }
                        ctx->npending = 0;
                    }
                    break;
                }
                launch_cohort(s, ctx, free_sl);
                launched = true;
            }
            if (ctx->npending) pending = true;
        }
        if (launched) continue;
        if (busy) {
            std::this_thread::sleep_for(std::chrono::microseconds(2));
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->inbox.empty() && !s->stop)
            s->cv_in.wait_for(lk, std::chrono::milliseconds(pending ? 1 : 50));
    }
}

}  // namespace

extern "C" {

int khop_server_create(const khop_server_opts *opts, khop_server **out) {
    if (!out) return KHOP_EINVAL;
    *out = nullptr;
    khop_server *s = new (std::nothrow) khop_server();
    if (!s) return KHOP_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.max_pending == 0) s->opts.max_pending = 1u << 20;
    int nsm = 0;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e);
    }
    s->grid_ctas = nsm;   // one CTA per SM: two cohort kernels fit side by side
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return KHOP_ENOMEM;
    }
    *out = s;
    return KHOP_OK;
}

int khop_submit(khop_server *s, khop_graph *g, uint32_t seed, uint32_t k, uint64_t *ticket) {
    if (!s || !g || !ticket) return KHOP_EINVAL;
    if ((uint64_t)seed >= g->n) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return KHOP_ESHUTDOWN;
    if (s->queued >= s->opts.max_pending) return KHOP_EBUSY;
    Request r{s->next_ticket++, g, seed, k, now_ns()};
    *ticket = r.ticket;
    s->submitted++;
    s->queued++;
    if (k == 0) {
        // nothing to traverse: complete at once
        khop_result res{r.ticket, 0ull, KHOP_OK, k, r.t_submit, now_ns()};
        s->outbox.push_back(res);
        s->completed++;
        s->queued--;
        s->cv_out.notify_all();
        return KHOP_OK;
    }
    s->inbox.push_back(r);
    s->cv_in.notify_one();
    return KHOP_OK;
}

int khop_submit_many(khop_server *s, khop_graph *g, const uint32_t *seeds, const uint32_t *ks,
                     uint32_t count, uint64_t *tickets) {
    if (!s || !g || (count && (!seeds || !ks || !tickets))) return KHOP_EINVAL;
    for (uint32_t i = 0; i < count; ++i)
        if ((uint64_t)seeds[i] >= g->n) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return KHOP_ESHUTDOWN;
    if (s->queued + count > s->opts.max_pending) return KHOP_EBUSY;
    const uint64_t t = now_ns();
    bool any = false;
    for (uint32_t i = 0; i < count; ++i) {
        Request r{s->next_ticket++, g, seeds[i], ks[i], t};
        tickets[i] = r.ticket;
        s->submitted++;
        s->queued++;
        if (ks[i] == 0) {
            khop_result res{r.ticket, 0ull, KHOP_OK, 0u, t, now_ns()};
            s->outbox.push_back(res);
            s->completed++;
            s->queued--;
            continue;
        }
        s->inbox.push_back(r);
        any = true;
    }
    if (any) s->cv_in.notify_one();
    s->cv_out.notify_all();
    return KHOP_OK;
}

int khop_poll(khop_server *s, khop_result *out, uint32_t max, uint32_t *nout, int64_t timeout_us) {
    if (!s || !nout || (max && !out)) return KHOP_EINVAL;
    *nout = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->outbox.empty() && timeout_us != 0) {
        auto ready = [s] { return !s->outbox.empty() || (s->stop && s->queued == 0); };
        if (timeout_us < 0) s->cv_out.wait(lk, ready);
        else s->cv_out.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    uint32_t n = 0;
    while (n < max && !s->outbox.empty()) {
        out[n++] = s->outbox.front();
        s->outbox.pop_front();
    }
    *nout = n;
    if (n == 0 && timeout_us != 0) return s->stop ? KHOP_ESHUTDOWN : KHOP_ETIMEDOUT;
    return KHOP_OK;
}

int khop_server_stats(khop_server *s, uint64_t *submitted, uint64_t *completed, uint64_t *steps,
                      uint64_t *batches_allocated) {
    if (!s) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (steps) *steps = s->steps;
    if (batches_allocated) *batches_allocated = s->slots_allocated;
    return KHOP_OK;
}

int khop_server_destroy(khop_server *s) {
    if (!s) return KHOP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests not yet seen by the worker
        for (auto &r : s->inbox) {
            khop_result res{r.ticket, ~0ull, KHOP_ESHUTDOWN, r.k, r.t_submit, now_ns()};
            s->outbox.push_back(res);
            s->completed++;
            s->queued--;
        }
        s->inbox.clear();
        s->cv_in.notify_all();
        s->cv_out.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return KHOP_OK;
}

}  // extern "C"
