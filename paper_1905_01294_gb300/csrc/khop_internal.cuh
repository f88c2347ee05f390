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

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
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

// Words of a software grid barrier for a cooperative launch.
struct BarrierWords {
    unsigned count;  // CTAs arrived at the current barrier
    unsigned gen;    // generation, bumped by the last arriver
};

// Grid-wide barrier over all CTAs of a cooperative launch.  Thread 0 of each
// CTA arrives with a release and waits with an acquire, so writes made before
// the barrier are visible to every thread after it.  The wait is bounded by
// `timeout_ns` of %globaltimer and by an iteration cap; on expiry (or if
// another CTA already flagged a timeout) it sets KHOP_DEVERR_TIMEOUT in *err
// and returns false, and the caller leaves the kernel.
__device__ __forceinline__ bool grid_barrier(BarrierWords *bw, unsigned *err, unsigned &epoch,
                                             uint64_t timeout_ns, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = epoch + 1u;
        int ok = 1;
        __threadfence();
        const unsigned arrived = atomicAdd(&bw->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            bw->count = 0u;
            __threadfence();
            st_release_u32(&bw->gen, target);
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint64_t spins = 0;
            while (ld_acquire_u32(&bw->gen) != target) {
                if ((++spins & 255u) == 0u) {
                    if (ld_volatile_u32(err) & KHOP_DEVERR_TIMEOUT) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > timeout_ns || spins > (1ull << 34)) {
                        atomicOr(err, (unsigned)KHOP_DEVERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        epoch = target;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// ---------------------------------------------------------------------------
// Host side

// Small device control block of a traversal state (zeroed before a launch).
struct CtlBlock {
    unsigned long long qpack[3];    // (queue items << ebits) | out-edge prefix, per round mod 3
    unsigned long long nnew[3];     // vertices discovered, per round mod 3
    unsigned long long scanned[3];  // in-edges examined by pull, per round mod 3
    BarrierWords bar;
    unsigned err;                   // sticky khop_device_error bits
    unsigned pad;
};
// Kernels address the counters as one array: qpack at [0,3), nnew at [3,6),
// scanned at [6,9).
static_assert(offsetof(CtlBlock, qpack) == 0 && offsetof(CtlBlock, nnew) == 24 &&
                  offsetof(CtlBlock, scanned) == 48,
              "CtlBlock counter layout");

// Bit-sliced (64-lane) batch state of a graph.
struct BatchState {
    uint64_t *V = nullptr;          // visited lanes per vertex [n]
    uint64_t *F[2] = {nullptr, nullptr};  // frontier lanes per vertex [n]
    uint32_t *Q[2] = {nullptr, nullptr};  // union-frontier vertices with out-edges
    void *Qpre[2] = {nullptr, nullptr};   // out-edge prefix per queue item (E)
    uint32_t *TF[2] = {nullptr, nullptr}; // first queue item of each push tile
    CtlBlock *ctl = nullptr;
    unsigned long long *lane_cnt = nullptr;  // [64] per-lane counts
    size_t bytes = 0;
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

    // plain single-query traversal state, device
    uint32_t *V = nullptr;
    uint32_t *F[3] = {nullptr, nullptr, nullptr};
    void *Qpre[2] = {nullptr, nullptr};
    void *Qrs[2] = {nullptr, nullptr};
    uint32_t *TF[2] = {nullptr, nullptr};
    uint64_t tf_cap = 0;
    khop::CtlBlock *ctl = nullptr;

    khop::BatchState batch;

    khop_tuning tune{};
    uint64_t timeout_ns = 2000000000ull;
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
int ensure_batch_state(khop_graph *g);                     // call under g->mu
int cooperative_grid(const void *kernel, int block, size_t smem, int want_per_sm, int num_sms,
                     int *grid);

// plain path (khop_plain.cu)
int plain_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint32_t k_all,
                 uint64_t nq, uint64_t *out, uint64_t *out_te, khop_query_stats *stats,
                 uint64_t *per_hop, uint32_t hop_stride, cudaStream_t st);

// batched path (khop_batch.cu)
int batch_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st);

}  // namespace khop
