// Continuous-batching request server for the k-hop count (khop_server_*).
//
// Requests (graph, seed, k) arrive from any host thread; a worker thread
// serves them on two kinds of slot, each with its own stream so that the
// slots' launches run side by side on the device.
//
// Heavy requests (k >= 3) are continuously batched at round granularity.  A
// rolling slot holds one 64-lane bit-sliced traversal on the device and runs
// it one round per launch (a step, see roll_kernel); lanes are independent,
// so every step advances each lane in use by one hop whatever its depth.
// Between steps the worker posts the result of every lane the step retired
// (its k-th round ran, or its frontier came out empty) the moment the step
// completes, and admits waiting requests into the free lanes, each with its
// own round counter: a request that arrives while a traversal runs joins it
// at the next round boundary.  A retired lane is reused once its marks are
// gone (see roll_kernel); when lanes run short the worker asks a step for a
// clearing sweep.  Deep traversals share their large middle rounds this way,
// so heavy slots are few: at most three per graph (max_batches permitting),
// each holding one depth class (k = 3, or k >= 4) so its lanes retire close
// together.
//
// Light requests (k <= 2) cost a few microseconds each on the single-query
// kernel, less than one round of a batch, so plain slots answer them in
// arrival order, up to kPlainBatch per persistent launch.
//
// Slots are allocated on demand, each only if free device memory (minus a
// margin) and the server's budget admit its state.  This is the GPU
// counterpart of the paper's thread pool serving many concurrent queries at
// low latency (Sec. II).
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

constexpr uint64_t kMarginBytes = 1ull << 30;
constexpr int kLanes = 64;
constexpr size_t kHeavySlots = 3;    // rolling slots per graph at most (three steps and a plain
                                     // launch are resident at once)
constexpr size_t kPlainSlots = 2;    // plain slots per graph at most
constexpr int kPlainBatch = 16;      // light requests per plain launch at most
constexpr uint32_t kAdmitWindow = 1; // default: a rolling slot admits while its lanes have run <= 1 round
constexpr int32_t kPlainHeavy = 2;   // default: heavy requests also take the single-query path while at
                                     // most this many wait (a traversal alone beats a batch's launches)

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

bool light(uint32_t k) { return k <= 2; }
// Queue of a request: 0 light, 1 heavy of depth 3, 2 deeper.  A rolling slot
// serves one depth class at a time, so its lanes finish at about the same
// round and the slot drains (and refills) without idling on a few deep lanes.
int queue_of(uint32_t k) { return light(k) ? 0 : (k <= 3 ? 1 : 2); }

struct Lane {
    bool used = false;     // holds a request
    bool dirty = false;    // retired, its visited marks not yet cleared (not reusable)
    bool fwait = false;    // retired, its bits still in the next frontier buffer (not reusable)
    uint64_t ret_round = 0;   // the state's round count when it retired
    Request req{};
    uint32_t rounds = 0;   // rounds completed
};

bool lane_free(const Lane &ln) { return !ln.used && !ln.dirty && !ln.fwait; }

// A rolling 64-lane batch.
struct Slot {
    BatchState st;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    RollResult *h_res = nullptr;   // mapped pinned memory, written by the step kernel
    RollResult *d_res = nullptr;   // its device address
    Lane lane[kLanes];
    int used = 0;                  // lanes in use
    int ndirty = 0;                // lanes waiting to be cleaned
    int queue = 0;                 // the heavy queue (1 or 2) it serves while lanes are in use
    bool busy = false;             // a step is in flight
    bool lost = false;             // that step was given up: its requests already failed
    bool reset = false;            // the next step starts from zeroed state
    uint64_t t_launch = 0;
    std::vector<std::pair<uint32_t, uint32_t>> admit;   // (lane, seed) for the next step
};

// Single-query path: one persistent launch answers a list of light requests.
struct PlainSlot {
    PlainState pst;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    uint32_t *d_q = nullptr, *h_q = nullptr;   // seeds[kPlainBatch], ks[kPlainBatch] (h_q pinned)
    uint64_t *h_out = nullptr, *d_out = nullptr;   // counts: mapped pinned memory the kernel writes
    std::vector<Request> reqs;     // the launch in flight
    bool busy = false, lost = false;
    uint64_t t_launch = 0;
};

struct GraphCtx {
    khop_graph *g = nullptr;
    std::deque<Request> pending[3];   // light, heavy of depth 3, deeper
    bool heavy_waiting() const { return !pending[1].empty() || !pending[2].empty(); }
    size_t heavy_pending() const { return pending[1].size() + pending[2].size(); }
    std::vector<Slot *> slots;
    std::vector<PlainSlot *> pslots;
    bool alloc_failed = false;       // the last rolling-slot allocation was refused
    bool palloc_failed = false;      // the last plain-slot allocation was refused
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
    std::atomic<int64_t> timeout_us{2000000};
    uint32_t admit_rounds = kAdmitWindow;
    int32_t plain_heavy = kPlainHeavy;
    uint64_t next_ticket = 1;
    khop_server_counters c{};
    uint64_t queued = 0;            // submitted and not yet completed
    uint64_t mem_used = 0;          // device bytes of the slots
    uint64_t lanes_busy = 0;        // worker-owned
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
    s->c.completed++;
    if (status == KHOP_ETIMEDOUT) s->c.timed_out++;
    s->queued--;
    s->cv_out.notify_all();
}

bool admit_memory(khop_server *s, uint64_t need) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return false;
    if ((uint64_t)fr < need + kMarginBytes) return false;
    return !(s->opts.mem_budget_bytes && s->mem_used + need > s->opts.mem_budget_bytes);
}

void free_slot(Slot *sl) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    free_batch_state(sl->st);
    if (sl->h_res) cudaFreeHost(sl->h_res);
    if (sl->ev) cudaEventDestroy(sl->ev);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
}

void free_pslot(PlainSlot *ps) {
    if (ps->stream) cudaStreamSynchronize(ps->stream);
    free_plain_state(ps->pst);
    cudaFree(ps->d_q);
    cudaFreeHost(ps->h_q);
    if (ps->h_out) cudaFreeHost(ps->h_out);
    if (ps->ev) cudaEventDestroy(ps->ev);
    if (ps->stream) cudaStreamDestroy(ps->stream);
    delete ps;
}

// A new rolling slot for ctx if the cap, memory and the budget admit it.
Slot *try_alloc_slot(khop_server *s, GraphCtx *ctx) {
    const uint64_t cap = std::min<uint64_t>(s->opts.max_batches ? s->opts.max_batches : kHeavySlots,
                                            kHeavySlots);
    if (ctx->slots.size() >= cap) return nullptr;
    const uint64_t need = batch_state_bytes(ctx->g) + 2 * ctx->g->n * sizeof(uint32_t) + 4096;   // + sink lists
    if (!admit_memory(s, need)) return nullptr;
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) return nullptr;
    uint64_t bytes = 0;
    bool ok;
    {
        // the slot belongs to the server, not to the graph's own accounting
        std::lock_guard<std::mutex> glk(ctx->g->mu);
        ok = alloc_batch_state(ctx->g, sl->st, &bytes, 1, true) == KHOP_OK;
        if (ok) ctx->g->device_bytes -= bytes;
    }
    ok = ok && cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&sl->h_res, sizeof(RollResult), cudaHostAllocMapped) == cudaSuccess;
    ok = ok && cudaHostGetDevicePointer((void **)&sl->d_res, sl->h_res, 0) == cudaSuccess;
    if (!ok) {
        free_slot(sl);
        return nullptr;
    }
    memset(sl->h_res, 0, sizeof(RollResult));
    s->mem_used += bytes;
    ctx->slots.push_back(sl);
    std::lock_guard<std::mutex> lk(s->mu);
    s->c.slots_allocated++;
    return sl;
}

// A new plain slot for ctx if the cap, memory and the budget admit it.
PlainSlot *try_alloc_pslot(khop_server *s, GraphCtx *ctx) {
    if (ctx->pslots.size() >= kPlainSlots) return nullptr;
    const uint64_t need = plain_state_bytes(ctx->g) + 4096;
    if (!admit_memory(s, need)) return nullptr;
    PlainSlot *ps = new (std::nothrow) PlainSlot();
    if (!ps) return nullptr;
    bool ok;
    {
        std::lock_guard<std::mutex> glk(ctx->g->mu);
        ok = alloc_plain_state(ctx->g, ps->pst) == KHOP_OK;
        if (ok) ctx->g->device_bytes -= ps->pst.bytes;
    }
    ok = ok && cudaStreamCreateWithFlags(&ps->stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ps->ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&ps->d_q, 2 * kPlainBatch * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ps->h_q, 2 * kPlainBatch * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&ps->h_out, kPlainBatch * sizeof(uint64_t), cudaHostAllocMapped) ==
                   cudaSuccess;
    ok = ok && cudaHostGetDevicePointer((void **)&ps->d_out, ps->h_out, 0) == cudaSuccess;
    if (!ok) {
        free_pslot(ps);
        return nullptr;
    }
    s->mem_used += ps->pst.bytes;
    ctx->pslots.push_back(ps);
    return ps;
}

// Fail every request holding a lane of sl and free the lanes; the slot
// restarts from zeroed state.
void fail_lanes(khop_server *s, Slot *sl, int status) {
    for (Lane &ln : sl->lane)
        if (ln.used) {
            post(s, ln.req, ~0ull, status);
            ln.used = false;
        }
    for (Lane &ln : sl->lane) ln.dirty = ln.fwait = false;
    sl->ndirty = 0;
    s->lanes_busy -= (uint64_t)sl->used;
    sl->used = 0;
    sl->admit.clear();
    sl->reset = true;
}

int free_lanes(const Slot *sl) {
    int c = 0;
    for (const Lane &ln : sl->lane) c += lane_free(ln);
    return c;
}

// Take waiting heavy requests of ctx into the free lanes of sl, oldest first,
// while the slot's traversal is in its admission window: a pull round skips
// a vertex's remaining in-edges only once every lane that needs the vertex
// found a parent, which lanes with small frontiers (just admitted) rarely
// do, so a traversal whose lanes went deep takes no new lanes until it drains.
void admit(khop_server *s, GraphCtx *ctx, Slot *sl) {
    int nfree = free_lanes(sl);
    if (nfree == 0 || !ctx->heavy_waiting()) return;
    if (sl->used == 0) {   // an empty slot serves the queue with the oldest request
        const bool a = !ctx->pending[1].empty(), b = !ctx->pending[2].empty();
        sl->queue = (a && (!b || ctx->pending[1].front().t_submit <= ctx->pending[2].front().t_submit)) ? 1 : 2;
    }
    // with one slot per graph (max_batches = 1) it serves both depth classes
    const bool shared = s->opts.max_batches == 1;
    if (!shared && ctx->pending[sl->queue].empty()) return;
    for (const Lane &ln : sl->lane)
        if (ln.used && ln.rounds > s->admit_rounds) return;
    const bool running = sl->used > 0;
    int l = 0;
    uint64_t joined = 0;
    while (nfree > 0) {
        std::deque<Request> *qp = &ctx->pending[sl->queue];
        if (shared) {   // the older head of the two queues
            std::deque<Request> &a = ctx->pending[1], &b = ctx->pending[2];
            if (a.empty() && b.empty()) break;
            qp = (!a.empty() && (b.empty() || a.front().t_submit <= b.front().t_submit)) ? &a : &b;
        }
        std::deque<Request> &q = *qp;
        if (q.empty()) break;
        while (!lane_free(sl->lane[l])) ++l;
        --nfree;
        Lane &ln = sl->lane[l];
        ln.used = true;
        ln.req = q.front();
        ln.rounds = 0;
        q.pop_front();
        sl->admit.emplace_back((uint32_t)l, ln.req.seed);
        sl->used++;
        s->lanes_busy++;
        joined += running;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->c.joined_running += joined;
    if (s->lanes_busy > s->c.max_lanes_busy) s->c.max_lanes_busy = s->lanes_busy;
}

// Launch the next step of sl: one round for every lane in use.
void launch_step(khop_server *s, GraphCtx *ctx, Slot *sl) {
    RollPlan p{};
    p.nadmit = (uint32_t)sl->admit.size();
    for (size_t t = 0; t < sl->admit.size(); ++t) {
        p.lane[t] = sl->admit[t].first;
        p.seed[t] = sl->admit[t].second;
    }
    sl->admit.clear();
    for (int l = 0; l < kLanes; ++l) {
        const Lane &ln = sl->lane[l];
        if (ln.dirty) p.clean |= 1ull << l;
        if (!ln.used) continue;
        p.act |= 1ull << l;
        if ((uint64_t)ln.rounds + 1 >= (uint64_t)ln.req.k) p.fin |= 1ull << l;
    }
    // lanes run short while requests wait: clear the retired lanes' marks now
    p.clean_dense = (p.clean != 0ull && ctx->heavy_waiting() && free_lanes(sl) <= kLanes / 2) ? 1u : 0u;
    p.pull_ok = 1u;   // lanes of a slot are within kAdmitWindow + 1 rounds of each other
    p.reset = sl->reset ? 1u : 0u;
    sl->reset = false;
    sl->h_res->done = 0ull;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->c.clean_steps += p.clean_dense;
        s->c.lane_steps += (uint64_t)__builtin_popcountll(p.act);
    }
    int rc = roll_launch(ctx->g, sl->st, p, sl->d_res, s->grid_ctas, sl->stream);
    if (rc == KHOP_OK) rc = cuda_status(cudaEventRecord(sl->ev, sl->stream));
    if (rc != KHOP_OK) {
        fail_lanes(s, sl, rc);
        return;
    }
    sl->busy = true;
    sl->lost = false;
    sl->t_launch = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    s->c.steps++;
}

// A step of sl completed: post the retired lanes, advance the others.
void finish_step(khop_server *s, Slot *sl) {
    sl->busy = false;
    if (sl->lost) {   // its requests failed already; the device state is abandoned
        sl->lost = false;
        for (Lane &ln : sl->lane) ln.used = ln.dirty = ln.fwait = false;
        sl->ndirty = 0;
        s->lanes_busy -= (uint64_t)sl->used;
        sl->used = 0;
        sl->reset = true;
        return;
    }
    const RollResult &r = *sl->h_res;
    if (r.done != 1ull) {
        fail_lanes(s, sl, KHOP_EDEVICE);
        return;
    }
    const unsigned long long retired = r.retired;
    uint64_t early = 0;
    for (int l = 0; l < kLanes; ++l) {
        Lane &ln = sl->lane[l];
        if (ln.dirty && ((r.cleaned >> l) & 1ull)) {
            ln.dirty = false;
            sl->ndirty--;
        }
        // stale frontier bits are gone once the buffer holding them was
        // consumed by a later round, or the state emptied
        if (ln.fwait && (r.idle || r.rdone > ln.ret_round)) ln.fwait = false;
        if (!ln.used) continue;
        if ((retired >> l) & 1ull) {
            if ((uint64_t)ln.rounds + 1 < (uint64_t)ln.req.k) ++early;
            post(s, ln.req, r.count[l], KHOP_OK);
            ln.used = false;
            if (r.count[l] != 0ull) {
                // it marked vertices besides its seed (whose mark is cleared already),
                // and its last discoveries are in the next frontier buffer
                ln.dirty = true;
                sl->ndirty++;
                ln.fwait = r.idle == 0ull;
                ln.ret_round = r.rdone;
            }
            sl->used--;
            s->lanes_busy--;
        } else {
            ln.rounds++;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->c.retired_early += early;
    s->c.gpu_step_ns += r.t_end_ns > r.t_start_ns ? r.t_end_ns - r.t_start_ns : 0ull;
    s->c.pull_steps += r.pulled;
}

// Launch the oldest waiting requests of queue `cls` of ctx on the plain slot ps.
void launch_plain(khop_server *s, GraphCtx *ctx, PlainSlot *ps, int cls) {
    std::deque<Request> &q = ctx->pending[cls];
    ps->reqs.clear();
    while (!q.empty() && (int)ps->reqs.size() < kPlainBatch) {
        ps->reqs.push_back(q.front());
        q.pop_front();
    }
    const size_t c = ps->reqs.size();
    for (size_t i = 0; i < c; ++i) {
        ps->h_q[i] = ps->reqs[i].seed;
        ps->h_q[kPlainBatch + i] = ps->reqs[i].k;
    }
    int rc = cuda_status(cudaMemcpyAsync(ps->d_q, ps->h_q, 2 * kPlainBatch * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, ps->stream));
    if (rc == KHOP_OK)
        rc = plain_launch_state(ctx->g, ps->pst, ps->d_q, ps->d_q + kPlainBatch, c, ps->d_out, s->grid_ctas,
                                ps->stream);   // (s->grid_ctas: half the SMs' CTA slots, see create)
    if (rc == KHOP_OK) rc = cuda_status(cudaEventRecord(ps->ev, ps->stream));
    if (rc != KHOP_OK) {
        for (const Request &r : ps->reqs) post(s, r, ~0ull, rc);
        ps->reqs.clear();
        return;
    }
    ps->busy = true;
    ps->lost = false;
    ps->t_launch = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    s->c.plain_launches++;
}

void finish_plain(khop_server *s, PlainSlot *ps, int status) {
    ps->busy = false;
    if (!ps->lost)
        for (size_t i = 0; i < ps->reqs.size(); ++i)
            post(s, ps->reqs[i], status == KHOP_OK ? ps->h_out[i] : ~0ull, status);
    ps->reqs.clear();
    ps->lost = false;
}

void worker_main(khop_server *s) {
    cudaSetDevice(s->device);
    std::vector<Request> incoming;
    uint64_t t_active = now_ns();   // the last time the worker had something to do
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
            ctx->pending[queue_of(r.k)].push_back(r);
        }
        incoming.clear();
        const uint64_t timeout_ns = (uint64_t)s->timeout_us.load() * 1000ull;
        // completions
        bool busy = false;
        for (auto &kv : s->graphs) {
            for (Slot *sl : kv.second->slots) {
                if (!sl->busy) continue;
                const cudaError_t q = cudaEventQuery(sl->ev);
                if (q == cudaSuccess) {
                    finish_step(s, sl);
                } else if (q == cudaErrorNotReady) {
                    busy = true;
                    if (!sl->lost && now_ns() - sl->t_launch > timeout_ns) {
                        // give the step up: its requests fail now; the slot is
                        // reused (from zeroed state) once the step completes
                        fail_lanes(s, sl, KHOP_ETIMEDOUT);
                        sl->lost = true;
                    }
                } else {
                    fail_lanes(s, sl, KHOP_ECUDA);
                    sl->busy = false;
                }
            }
            for (PlainSlot *ps : kv.second->pslots) {
                if (!ps->busy) continue;
                const cudaError_t q = cudaEventQuery(ps->ev);
                if (q == cudaSuccess) {
                    finish_plain(s, ps, KHOP_OK);
                } else if (q == cudaErrorNotReady) {
                    busy = true;
                    if (!ps->lost && now_ns() - ps->t_launch > timeout_ns) {
                        for (const Request &r : ps->reqs) post(s, r, ~0ull, KHOP_ETIMEDOUT);
                        ps->lost = true;   // reused once the launch completes
                    }
                } else {
                    finish_plain(s, ps, KHOP_ECUDA);
                }
            }
        }
        if (stopping) {
            for (auto &kv : s->graphs) {
                GraphCtx *ctx = kv.second;
                // launches are bounded (every device wait is); what they do not
                // finish fails below
                for (Slot *sl : ctx->slots)
                    if (sl->busy) {
                        cudaStreamSynchronize(sl->stream);
                        finish_step(s, sl);
                    }
                for (PlainSlot *ps : ctx->pslots)
                    if (ps->busy) {
                        const cudaError_t e = cudaStreamSynchronize(ps->stream);
                        finish_plain(s, ps, e == cudaSuccess ? KHOP_OK : KHOP_ECUDA);
                    }
                for (Slot *sl : ctx->slots) {
                    fail_lanes(s, sl, KHOP_ESHUTDOWN);
                    free_slot(sl);
                }
                for (PlainSlot *ps : ctx->pslots) free_pslot(ps);
                for (auto &q : ctx->pending)
                    for (auto &r : q) post(s, r, ~0ull, KHOP_ESHUTDOWN);
                delete ctx;
            }
            s->graphs.clear();
            return;
        }
        // launches: every idle plain slot takes the oldest light requests;
        // every rolling slot at a step boundary admits heavy requests into its
        // free lanes and runs its next step; requests left over get new slots
        // while the caps, memory and the budget allow
        bool launched = false;
        for (auto &kv : s->graphs) {
            GraphCtx *ctx = kv.second;
            // light requests first; heavy ones too while only a few wait
            const auto plain_cls = [&]() {
                if (!ctx->pending[0].empty()) return 0;
                if (ctx->heavy_waiting() && s->plain_heavy >= 0 && ctx->heavy_pending() <= (size_t)s->plain_heavy) {
                    const bool a = !ctx->pending[1].empty(), b = !ctx->pending[2].empty();
                    return (a && (!b || ctx->pending[1].front().t_submit <= ctx->pending[2].front().t_submit)) ? 1 : 2;
                }
                return -1;
            };
            for (PlainSlot *ps : ctx->pslots) {
                const int c = plain_cls();
                if (c < 0) break;
                if (!ps->busy) {
                    launch_plain(s, ctx, ps, c);
                    launched = true;
                }
            }
            while (plain_cls() >= 0 && !ctx->palloc_failed) {
                PlainSlot *ps = try_alloc_pslot(s, ctx);
                if (!ps) {
                    ctx->palloc_failed = true;
                    break;
                }
                launch_plain(s, ctx, ps, plain_cls());
                launched = true;
            }
            for (Slot *sl : ctx->slots) {
                if (sl->busy) continue;
                admit(s, ctx, sl);
                // all of its lanes wait for cleaning while requests wait: a
                // step that only clears their marks
                const bool need_clean = sl->ndirty > 0 && sl->used == 0 && free_lanes(sl) <= kLanes / 2 &&
                                        ctx->heavy_waiting();
                if (sl->used > 0 || need_clean) {
                    launch_step(s, ctx, sl);
                    launched = true;
                }
            }
            while (ctx->heavy_waiting() && !ctx->alloc_failed) {
                Slot *sl = try_alloc_slot(s, ctx);
                if (!sl) {
                    ctx->alloc_failed = true;
                    break;
                }
                admit(s, ctx, sl);
                launch_step(s, ctx, sl);
                launched = true;
            }
            // requests that no slot of their kind could ever run fail
            if (ctx->pslots.empty() && ctx->palloc_failed) {
                for (auto &r : ctx->pending[0]) post(s, r, ~0ull, KHOP_ENOMEM);
                ctx->pending[0].clear();
            }
            if (ctx->slots.empty() && ctx->alloc_failed) {
                for (int qi = 1; qi <= 2; ++qi) {
                    for (auto &r : ctx->pending[qi]) post(s, r, ~0ull, KHOP_ENOMEM);
                    ctx->pending[qi].clear();
                }
            }
            if (ctx->pending[0].empty()) ctx->palloc_failed = false;   // try again next time
            if (!ctx->heavy_waiting()) ctx->alloc_failed = false;
        }
        // poll again at once while launches run or requests came lately: a
        // timed sleep or a condition-variable wake-up here costs tens of
        // microseconds, longer than a light request's whole launch
        const uint64_t now = now_ns();
        if (launched || busy) t_active = now;
        if (launched) continue;
        if (busy || now - t_active < 200000ull) {
            std::this_thread::yield();
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->inbox.empty() && !s->stop) s->cv_in.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

extern "C" {

int khop_server_create(const khop_server_opts *opts, khop_server **out) {
    if (!out) return KHOP_EINVAL;
    *out = nullptr;
    if (opts && opts->wait_timeout_us < 0) return KHOP_EINVAL;
    khop_server *s = new (std::nothrow) khop_server();
    if (!s) return KHOP_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.max_pending == 0) s->opts.max_pending = 1u << 20;
    s->timeout_us = s->opts.wait_timeout_us > 0 ? s->opts.wait_timeout_us : 2000000;
    s->admit_rounds = s->opts.admit_rounds ? s->opts.admit_rounds : kAdmitWindow;
    s->plain_heavy = s->opts.plain_heavy ? s->opts.plain_heavy : kPlainHeavy;
    int nsm = 0;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e);
    }
    // every launch of the server (steps, plain launches) on half the SMs'
    // worth of CTAs: four of them are resident at once (two per SM), so a
    // light request's launch never waits for a traversal's step to end
    s->grid_ctas = std::max(1, nsm / 2);
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return KHOP_ENOMEM;
    }
    *out = s;
    return KHOP_OK;
}

int khop_server_set_wait_timeout(khop_server *s, int64_t wait_timeout_us) {
    if (!s || wait_timeout_us < 0) return KHOP_EINVAL;
    s->timeout_us = wait_timeout_us > 0 ? wait_timeout_us : 2000000;
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
    s->c.submitted++;
    s->queued++;
    if (k == 0) {
        // nothing to traverse: complete at once
        khop_result res{r.ticket, 0ull, KHOP_OK, k, r.t_submit, now_ns()};
        s->outbox.push_back(res);
        s->c.completed++;
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
        s->c.submitted++;
        s->queued++;
        if (ks[i] == 0) {
            khop_result res{r.ticket, 0ull, KHOP_OK, 0u, t, now_ns()};
            s->outbox.push_back(res);
            s->c.completed++;
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
    if (submitted) *submitted = s->c.submitted;
    if (completed) *completed = s->c.completed;
    if (steps) *steps = s->c.steps;
    if (batches_allocated) *batches_allocated = s->c.slots_allocated;
    return KHOP_OK;
}

int khop_server_counters_get(khop_server *s, khop_server_counters *out) {
    if (!s || !out) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->c;
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
            s->c.completed++;
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
