// Internal declarations of libkhop (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cstddef>
#include <mutex>
#include <cuda_runtime.h>

#include "khop.h"

#define KHOP_VERSION_NUM 10000  // 1.0.0

namespace khop {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Asynchronous global -> shared copy of N bytes (4, 8 or 16; both addresses
// N-aligned), completed by cp_async_wait_all() of the same thread.
template <int N>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Wait until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ void prefetch_l2(const T *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p) {
    return *(const volatile unsigned *)p;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Word of a software grid barrier for a cooperative launch, alone on its
// 128-byte line.
struct BarrierWords {
    unsigned count;          // sense-reversing arrival counter
    unsigned pad[31];
};

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Grid-wide barrier over all CTAs of a cooperative launch: a sense-reversing
// counter.  Every CTA adds to one 32-bit word -- CTA 0 adds 2^31 - (G - 1),
// the other G - 1 CTAs add 1 -- so the barrier's additions total exactly 2^31:
// the top bit flips when, and only when, the last CTA has arrived, and the low
// bits return to where they were (no reset is ever needed).  Each CTA's
// thread 0 keeps the top bit it expects in `sense` (read once at kernel start
// with barrier_sense(): the bit cannot flip before every CTA, this one
// included, has arrived).  After a CTA-wide __syncthreads, thread 0 publishes
// the CTA's writes with a gpu-scope release reduction (no reply to wait for)
// and polls the word with relaxed loads until the top bit flips, then fences
// (acquire) before the rest of the CTA reads what the other CTAs wrote.  The wait is
// bounded by `timeout_ns` of %globaltimer and by an iteration cap; on expiry
// (or if another CTA already flagged a timeout) it sets KHOP_DEVERR_TIMEOUT in
// *err and returns false, and the caller leaves the kernel.
// If `post_n` > 0, thread 0 copies post_n 64-bit words from `post_src`
// (global, written before the barrier) to `post_dst` (shared) after the
// wait, so the rest of the CTA reads them from shared memory.
// `overlap(t, nt)` runs on threads 32 .. blockDim.x - 1 (t = threadIdx.x - 32,
// nt = blockDim.x - 32) while thread 0 waits: work that needs no ordering
// against the barrier (prefetches).  `pre()` runs on every thread of the CTA
// after its arrival and before its wait (a split barrier): work that reads
// only data no CTA writes and writes only this CTA's shared memory.
__device__ __forceinline__ unsigned barrier_sense(const BarrierWords *bw) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&bw->count) : "memory");
    return v & 0x80000000u;
}

// What thread 0 of a CTA keeps across the grid barriers of a launch: the
// sense it expects next, and (for testing failure detection) a countdown:
// when `absent_left` is non-zero, the CTA does not arrive at its
// absent_left-th barrier -- it waits for the others to give up instead -- so
// that their bounded wait runs out the way it would if a CTA were lost.
struct BarState {
    unsigned sense;
    unsigned absent_left;
};

// Thread 0's state at kernel start: the current sense; the last CTA of the
// grid gets the countdown `absent_at` (0 = arrive at every barrier).
__device__ __forceinline__ BarState barrier_start(const BarrierWords *bw, unsigned absent_at) {
    BarState b{0u, 0u};
    if (threadIdx.x == 0) {
        b.sense = barrier_sense(bw);
        if (blockIdx.x == gridDim.x - 1) b.absent_left = absent_at;
    }
    return b;
}

// Beamer's direction tests (x * c > y, x * c < y for a tuning factor c) in
// integer arithmetic: c is carried in 1/65536 units and both sides are
// compared as 128-bit products.  The per-round decisions thus need no FP64,
// whose rate on this part is a small fraction of the integer rate (a handful
// of double operations by every warp of a CTA cost about a microsecond).
inline uint64_t factor_fx16(float c) {
    if (!(c > 0.0f)) return 0ull;
    const double v = (double)c * 65536.0 + 0.5;
    return v >= 4.0e18 ? 4000000000000000000ull : (uint64_t)v;
}
__device__ __forceinline__ bool fx_gt(uint64_t x, uint64_t c_fx, uint64_t y) {
    return (unsigned __int128)x * c_fx > ((unsigned __int128)y << 16);
}
__device__ __forceinline__ bool fx_lt(uint64_t x, uint64_t c_fx, uint64_t y) {
    return (unsigned __int128)x * c_fx < ((unsigned __int128)y << 16);
}

struct NoOverlap {
    __device__ void operator()(unsigned, unsigned) const {}
};

struct NoPre {
    __device__ void operator()() const {}
};

template <typename Overlap = NoOverlap, typename Pre = NoPre>
__device__ __forceinline__ bool grid_barrier(BarrierWords *bw, unsigned *err, int *s_flag,
                                             BarState &bs,
                                             const unsigned long long *post_src = nullptr,
                                             unsigned long long *post_dst = nullptr,
                                             int post_n = 0, uint64_t timeout_ns = 2000000000ull,
                                             const Overlap &overlap = Overlap(),
                                             const Pre &pre = Pre()) {
    __syncthreads();
    bool absent = false;
    if (threadIdx.x == 0) {
        if (bs.absent_left != 0u && --bs.absent_left == 0u) {
            absent = true;   // stays away: the others' wait must run out
        } else {
            const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&bw->count), "r"(add)
                         : "memory");
            bs.sense ^= 0x80000000u;
        }
    }
    pre();
    if (threadIdx.x == 0 && absent) {
        // Wait (sleeping) until another CTA records the timeout, bounded by
        // twice the limit plus a millisecond, then leave like the others.
        const uint64_t t0 = globaltimer_ns();
        while (!(ld_volatile_u32(err) & KHOP_DEVERR_TIMEOUT) &&
               globaltimer_ns() - t0 < 2ull * timeout_ns + 1000000ull)
            __nanosleep(1000);
        atomicOr(err, (unsigned)KHOP_DEVERR_TIMEOUT);
        *s_flag = 0;
    } else if (threadIdx.x == 0) {
        const unsigned sense = bs.sense;
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        uint64_t spins = 0;
        while ((ld_relaxed_u32(&bw->count) & 0x80000000u) != sense) {
            ++spins;
            if ((spins & 255u) == 0u) {
                if (ld_volatile_u32(err) & KHOP_DEVERR_TIMEOUT) { ok = 0; break; }
                if (globaltimer_ns() - t0 > timeout_ns || spins > (1ull << 32)) {
                    atomicOr(err, (unsigned)KHOP_DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel_gpu();   // acquire: the flip was read relaxed
        for (int i = 0; i < post_n; ++i) post_dst[i] = ld_relaxed_u64(post_src + i);
        *s_flag = ok;
    } else if (threadIdx.x >= 32) {
        overlap(threadIdx.x - 32u, blockDim.x - 32u);
    }
    __syncthreads();
    return *s_flag != 0;
}

// ---------------------------------------------------------------------------
// Host side

// Per-round counters of a traversal, one slot per round mod 3.
struct RoundSlot {
    unsigned long long qpack;     // (queue items << ebits) | out-edge prefix of the queue
    unsigned long long nnew;      // vertices discovered
    unsigned long long scanned;   // in-edges examined by pull
    unsigned long long mf;        // out-edges of the vertices discovered
    unsigned long long unv;       // vertices a pull round had to examine
    unsigned long long defer[2];  // batched pull: deferred in-lists, their chunks
    unsigned long long seen;      // rolling batch: lanes that discovered a vertex
    unsigned long long sinks;     // rolling batch: discovered vertices without out-edges
    unsigned long long pad[7];
};
constexpr int kSlotWords = sizeof(RoundSlot) / 8;

// Small device control block of a traversal state (zeroed before a launch,
// except `err`).
struct CtlBlock {
    RoundSlot slot[3];
    unsigned long long pad[4];      // batched path: [0] batches, [1] algorithmic bytes,
                                    // [2] rounds, [3] pull rounds
    unsigned long long handoff[16]; // plain path: state left by the one-CTA rounds
    BarrierWords bar;
    // Kept across launches (a launch clears only what comes before `err`):
    unsigned err;                   // sticky khop_device_error bits
    unsigned dirty;                 // batched state may be dirty (a launch did not finish)
    unsigned long long rdone;       // batched: rounds run so far (frontier buffer rotation)
    uint32_t one_q[2];              // plain path: (seed, k) of a single-query call
    unsigned long long one_out;     //   and its count
    unsigned pad2[24];
};

// Plain single-query traversal state (one query at a time).
struct PlainState {
    uint32_t *V = nullptr, *V2 = nullptr;         // visited bitmaps (queries alternate)
    uint32_t *F[3] = {nullptr, nullptr, nullptr}; // frontier bitmaps, rotating per round
    void *Qpre[2] = {nullptr, nullptr};           // queue: out-edge prefix (E)
    void *Qrs[2] = {nullptr, nullptr};            // queue: row start (E)
    uint32_t *TF[2] = {nullptr, nullptr};         // first queue item of each push tile
    CtlBlock *ctl = nullptr;
    uint64_t bytes = 0;
};

// Bit-sliced batch state of a graph: 64 * lw lanes per vertex word (lw 64-bit
// words per vertex in V, F, and the deferred-in-list lane masks).
struct BatchState {
    uint64_t *V = nullptr;                        // visited lanes per vertex [n]
    uint32_t *S[2] = {nullptr, nullptr};          // rolling batch: discovered sinks per round [n]
    uint64_t *F[3] = {nullptr, nullptr, nullptr}; // frontier lanes per vertex [n], rotating
    uint32_t *Q[2] = {nullptr, nullptr};          // union-frontier vertices with out-edges
    void *Qpre[2] = {nullptr, nullptr};           // out-edge prefix per queue item (E)
    uint32_t *TF[2] = {nullptr, nullptr};         // first queue item of each push tile
    CtlBlock *ctl = nullptr;
    unsigned long long *part = nullptr;           // per-CTA lane counts [2][part_rows][64]
    uint64_t part_rows = 0;
    uint32_t *order = nullptr;                    // batch lane table (query indices)
    uint64_t order_cap = 0;
    // pull rounds: vertices whose in-lists are finished in chunks
    uint32_t *hv = nullptr;
    void *hend = nullptr;                         // E
    unsigned long long *hneed = nullptr, *hacc = nullptr;
    uint64_t hcap = 0;
    uint32_t *ch_item = nullptr;
    void *ch_start = nullptr;                     // E
    uint64_t ccap = 0;
    size_t bytes = 0;
    int lw = 1;
};

// One step of a rolling 64-lane batch (the request server's continuous
// batching): the host's plan, passed by value as a kernel argument, and the
// step's outcome, written by the kernel into mapped pinned host memory.
struct RollPlan {
    uint32_t nadmit;              // lanes admitted at the start of this step
    uint32_t reset;               // 1: start from zeroed state (after a step that was given up)
    unsigned long long act;       // lanes that run this round (admitted lanes included)
    unsigned long long fin;       // lanes whose k is reached with this round
    unsigned long long clean;     // retired lanes whose visited marks are still to be cleared
    uint32_t clean_dense;         // 1: clear them everywhere now (a V sweep)
    uint32_t pull_ok;             // 0: the round always pushes (see roll_kernel)
    uint32_t lane[64];            // admission t: lane[t] starts seed[t] (its q_0 = {seed})
    uint32_t seed[64];
};

struct RollResult {
    unsigned long long retired;   // lanes whose count is final after this step
    unsigned long long cleaned;   // lanes of plan.clean whose visited marks are all gone
    unsigned long long rdone;     // rounds run by the state so far (after this step)
    unsigned long long idle;      // 1: no lane continues; every frontier buffer is zero
    unsigned long long union_nf;  // vertices in the union frontier after the round
    unsigned long long bytes;     // algorithmic bytes of the round
    unsigned long long pulled;    // 1 if the round ran as a pull
    unsigned long long t_start_ns, t_end_ns;   // %globaltimer at the step's start and end (CTA 0)
    unsigned long long done;      // written last: the step completed
    unsigned long long count[64]; // the retired lanes' counts
};

}  // namespace khop

struct khop_graph {
    uint64_t n = 0, nnz = 0;
    int ewidth = 4;        // bytes of an internal edge offset (4 if nnz < 2^32, else 8)
    bool symmetric = false;
    int device = 0, num_sms = 0;
    uint32_t nw = 0;       // 32-bit words of a vertex bitmap
    uint32_t ebits = 32;   // bits of the out-edge prefix in a packed queue counter

    // CSR (out-edges) and CSC (in-edges), device
    void *rp = nullptr;
    uint32_t *ci = nullptr;
    void *cp = nullptr;
    uint32_t *ri = nullptr;

    uint32_t *noin = nullptr;               // bit set: vertex has no in-edge
    uint64_t n_noin = 0;                    // vertices without in-edges
    uint64_t tf_cap = 0;                    // push-tile map entries
    khop::PlainState plain;                 // plain single-query traversal state

    khop::BatchState batch;                 // 64 lanes
    khop::BatchState batch2;                // 128 lanes (allocated on first use)
    khop::BatchState batch4;                // 256 lanes (allocated on first use)
    int last_lw = 1;                        // lane width of the last batched call

    khop_tuning tune{};
    // khop_mxv: the in-lists longer than kMxvLong, cut into chunks (built on first use)
    uint32_t *mxv_cv = nullptr;             // vertex of each chunk
    unsigned long long *mxv_cs = nullptr;   // first in-edge of each chunk
    uint64_t mxv_nch = 0;                   // chunks
    bool mxv_ready = false;
    uint64_t timeout_ns = 2000000000ull;   // bound of every device wait (grid barriers)
    unsigned absent_at = 0;                // testing: see khop_graph_test_absent_cta
    uint64_t device_bytes = 0;

    std::mutex mu;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
};

namespace khop {

// helpers implemented in khop_graph.cu
int cuda_status(cudaError_t e);
int order_after_previous(khop_graph *g, cudaStream_t s);   // call under g->mu
int mark_done(khop_graph *g, cudaStream_t s);              // call under g->mu
int ensure_batch_state(khop_graph *g, int lw = 1);         // call under g->mu
// a standalone state; `sinks`: with the rolling batch's sink lists
int alloc_batch_state(khop_graph *g, BatchState &b, uint64_t *bytes, int lw = 1, bool sinks = false);
int alloc_plain_state(khop_graph *g, PlainState &p);
void free_plain_state(PlainState &p);
void free_batch_state(BatchState &b);
uint64_t batch_state_bytes(const khop_graph *g);
uint64_t plain_state_bytes(const khop_graph *g);
int cooperative_grid(const void *kernel, int block, size_t smem, int want_per_sm, int num_sms,
                     int *grid);
// Open `kernel` to `smem` bytes of dynamic shared memory (once per device)
// and give the grid of a cooperative launch (resident CTAs per SM, capped by
// want_per_sm if > 0, times num_sms); both answers are cached, so a launch
// path pays for the runtime queries only once.
int launch_shape(const void *kernel, int block, size_t smem, int want_per_sm, int num_sms, int *grid);

// plain path (khop_plain.cu)
// keep_visited: every query runs on the grid path, so that after a launch of
// one query the visited bitmap plain.V holds its whole neighbourhood.
// levels (or null): levels[w] = r for every w discovered in round r.
int plain_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint32_t k_all,
                 uint64_t nq, uint64_t *out, uint64_t *out_te, khop_query_stats *stats,
                 uint64_t *per_hop, uint32_t hop_stride, cudaStream_t st,
                 bool keep_visited = false, int32_t *levels = nullptr);
// The same on a standalone state, with at most grid_ctas CTAs (0 = fill the GPU).
int plain_launch_state(khop_graph *g, PlainState &ps, const uint32_t *seeds, const uint32_t *ks,
                       uint64_t nq, uint64_t *out, int grid_ctas, cudaStream_t st);

// batched path (khop_batch.cu); lw = 1, 2 or 4 (64, 128 or 256 lanes per traversal)
int batch_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st, int lw = 1);
// One step of the rolling 64-lane batch held in `bs` (its results go to
// `res`, device-visible), on at most grid_ctas CTAs.
int roll_launch(khop_graph *g, BatchState &bs, const RollPlan &plan, RollResult *res,
                int grid_ctas, cudaStream_t st);

}  // namespace khop
