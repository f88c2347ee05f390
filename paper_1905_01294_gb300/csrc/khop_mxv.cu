// Masked matrix-vector product over a semiring (khop_mxv): y = A^T x, i.e.
//     y[v] = (+)_{u : A[u][v] = 1}  x[u] (x) 1
// for the vertices v the mask selects, and the (+)-identity elsewhere.  The
// paper's Sec. II runs every traversal as such sparse products; the k-hop
// count is the (OR, AND) case iterated with the visited set as the
// complemented mask.  Supported semirings (A's entries are 1):
//   OR_AND      y[v] = 1 if some in-neighbour has x[u] != 0, else 0
//   PLUS_TIMES  y[v] = sum of x[u] over the in-edges, mod 2^64 (iterated from
//               e_s it counts walks)
//   MIN_SECOND  y[v] = min of x[u] over the in-edges (UINT64_MAX = none); with
//               x[u] = u on a frontier it gives BFS parents
//   MAX_SECOND  y[v] = max of x[u] over the in-edges (0 = none)
// The sums run over the stored in-edges, so a duplicated edge adds twice.
// One warp takes 32 consecutive vertices (a coalesced read of their column
// offsets and mask word); each lane folds its vertex's first in-edges itself
// (four index loads in flight), then the warp folds the lists of up to
// kMxvLong edges one vertex at a time, 32 lanes wide, and reduces across
// lanes with shuffles.  Longer in-lists (the hubs of a power-law graph, which
// hold much of the edges) are cut into chunks of at most kMxvChunk edges,
// listed once per graph; a second kernel folds each chunk with one warp
// (coalesced index loads, eight in flight per lane) and combines the warp's
// result into y[v] with one atomic, so no warp walks a hub's list alone and
// no CTA waits on another's barrier.  OR_AND stops a list at its first hit.
#include <algorithm>

#include "khop_internal.cuh"

namespace khop {
namespace {

template <int SR>
struct Semiring;
template <>
struct Semiring<KHOP_SR_OR_AND> {
    static constexpr unsigned long long zero = 0ull;
    __device__ static unsigned long long add(unsigned long long a, unsigned long long b) { return a | (b != 0ull); }
    __device__ static unsigned long long join(unsigned long long a, unsigned long long b) { return a | b; }
    __device__ static bool done(unsigned long long a) { return a != 0ull; }
    __device__ static void combine(unsigned long long *p, unsigned long long a) { atomicOr(p, a); }
};
template <>
struct Semiring<KHOP_SR_PLUS_TIMES> {
    static constexpr unsigned long long zero = 0ull;
    __device__ static unsigned long long add(unsigned long long a, unsigned long long b) { return a + b; }
    __device__ static unsigned long long join(unsigned long long a, unsigned long long b) { return a + b; }
    __device__ static bool done(unsigned long long) { return false; }
    __device__ static void combine(unsigned long long *p, unsigned long long a) { atomicAdd(p, a); }
};
template <>
struct Semiring<KHOP_SR_MIN_SECOND> {
    static constexpr unsigned long long zero = ~0ull;
    __device__ static unsigned long long add(unsigned long long a, unsigned long long b) { return b < a ? b : a; }
    __device__ static unsigned long long join(unsigned long long a, unsigned long long b) { return b < a ? b : a; }
    __device__ static bool done(unsigned long long) { return false; }
    __device__ static void combine(unsigned long long *p, unsigned long long a) { atomicMin(p, a); }
};
template <>
struct Semiring<KHOP_SR_MAX_SECOND> {
    static constexpr unsigned long long zero = 0ull;
    __device__ static unsigned long long add(unsigned long long a, unsigned long long b) { return b > a ? b : a; }
    __device__ static unsigned long long join(unsigned long long a, unsigned long long b) { return b > a ? b : a; }
    __device__ static bool done(unsigned long long) { return false; }
    __device__ static void combine(unsigned long long *p, unsigned long long a) { atomicMax(p, a); }
};

#ifndef KHOP_MXV_LONG
#define KHOP_MXV_LONG 256
#endif
#ifndef KHOP_MXV_CHUNK
#define KHOP_MXV_CHUNK 1024
#endif
constexpr int kLaneList = 32;                   // in-edges a lane folds alone before the warp helps
constexpr uint64_t kMxvLong = KHOP_MXV_LONG;    // longer in-lists go to the chunk kernel
constexpr uint64_t kMxvChunk = KHOP_MXV_CHUNK;  // in-edges per chunk (one warp's task)
constexpr int kChunkLoads = 8;                  // index loads in flight per lane

template <typename E, int SR>
__global__ void __launch_bounds__(256) mxv_kernel(const E *cp, const uint32_t *ri, const unsigned long long *x,
                                                  const uint32_t *mask, unsigned comp, uint64_t n, uint64_t nw,
                                                  unsigned long long *y, unsigned long long *scanned_out) {
    using S = Semiring<SR>;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t scanned = 0;
    for (uint64_t i = gwarp; i < nw; i += nwarps) {
        const uint64_t v = (i << 5) + (uint64_t)lane;
        bool on = v < n;
        if (on && mask) on = (((mask[i] >> lane) & 1u) ^ comp) != 0u;
        E b = 0, e = 0;
        if (on) {
            b = cp[v];
            e = cp[v + 1];
            if ((uint64_t)(e - b) > kMxvLong) on = false;   // the chunk kernel folds it
        }
        unsigned long long acc = S::zero;
        E pos = b;
        const E lend = min(e, b + (E)kLaneList);
        while (__any_sync(FULL, on && pos < lend && !S::done(acc))) {
            if (on && pos < lend && !S::done(acc)) {
                uint32_t u[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) u[t] = pos + t < lend ? ri[pos + t] : 0xffffffffu;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (u[t] != 0xffffffffu) acc = S::add(acc, x[u[t]]);
                const E took = min((E)4, lend - pos);
                pos += took;
                scanned += (uint64_t)took;
            }
        }
        unsigned todo = __ballot_sync(FULL, on && pos < e && !S::done(acc));
        while (todo) {
            const int L = __ffs(todo) - 1;
            todo &= todo - 1u;
            const E lb = __shfl_sync(FULL, pos, L), le = __shfl_sync(FULL, e, L);
            unsigned long long part = S::zero;
            for (E c = lb; c < le; c += 64) {
                const E i0 = c + (E)lane, i1 = c + 32 + (E)lane;
                const uint32_t u0 = i0 < le ? ri[i0] : 0xffffffffu;
                const uint32_t u1 = i1 < le ? ri[i1] : 0xffffffffu;
                if (u0 != 0xffffffffu) part = S::add(part, x[u0]);
                if (u1 != 0xffffffffu) part = S::add(part, x[u1]);
                if (lane == 0) scanned += (uint64_t)min((E)64, le - c);
                if (SR == KHOP_SR_OR_AND && __any_sync(FULL, part != 0ull)) break;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part = S::join(part, __shfl_xor_sync(FULL, part, o));
            if (lane == L) acc = S::join(acc, part);
        }
        if (v < n) y[v] = on ? acc : S::zero;
    }
    scanned = warp_sum(scanned);
    if (lane == 0 && scanned) atomicAdd(scanned_out, (unsigned long long)scanned);
}

// The long in-lists, chunk by chunk: one warp folds a chunk (kChunkLoads
// coalesced index loads in flight per lane), reduces across its lanes and
// combines the result into y[v] atomically (y[v] was set to the identity by
// mxv_kernel, earlier on the same stream).
template <typename E, int SR>
__global__ void __launch_bounds__(256) mxv_chunk_kernel(const E *cp, const uint32_t *ri, const unsigned long long *x,
                                                        const uint32_t *mask, unsigned comp, const uint32_t *cv,
                                                        const unsigned long long *cs, uint64_t nch,
                                                        unsigned long long *y, unsigned long long *scanned_out) {
    using S = Semiring<SR>;
    constexpr uint64_t kStep = 32 * kChunkLoads;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t scanned = 0;
    for (uint64_t c = gwarp; c < nch; c += nwarps) {
        const uint32_t v = cv[c];
        // lane 0 decides for the warp: a vertex outside the mask, or (OR_AND) one
        // another chunk has already set, is skipped
        int skip = 0;
        if (lane == 0) {
            skip = mask && ((((mask[v >> 5] >> (v & 31)) & 1u) ^ comp) == 0u);
            if (SR == KHOP_SR_OR_AND && !skip) skip = *(volatile unsigned long long *)&y[v] != 0ull;
        }
        if (__shfl_sync(FULL, skip, 0)) continue;
        const uint64_t b = cs[c];
        const uint64_t e = min(b + kMxvChunk, (uint64_t)cp[v + 1]);
        unsigned long long acc = S::zero;
        for (uint64_t q = b; q < e; q += kStep) {
            uint32_t u[kChunkLoads];
#pragma unroll
            for (int t = 0; t < kChunkLoads; ++t) {
                const uint64_t p = q + (uint64_t)(t * 32 + lane);
                u[t] = p < e ? ri[p] : 0xffffffffu;
            }
#pragma unroll
            for (int t = 0; t < kChunkLoads; ++t)
                if (u[t] != 0xffffffffu) acc = S::add(acc, x[u[t]]);
            scanned += min(kStep, e - q);
            if (SR == KHOP_SR_OR_AND && __any_sync(FULL, acc != 0ull)) break;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = S::join(acc, __shfl_xor_sync(FULL, acc, o));
        if (lane == 0 && acc != S::zero) S::combine(&y[v], acc);
    }
    if (lane == 0 && scanned) atomicAdd(scanned_out, (unsigned long long)scanned);
}

// Chunks of the in-lists longer than kMxvLong, in any order.
template <typename E>
__global__ void mxv_plan_kernel(const E *cp, uint64_t n, uint32_t *cv, unsigned long long *cs, uint64_t cap,
                                unsigned long long *count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint64_t b = cp[v], d = (uint64_t)cp[v + 1] - b;
        if (d <= kMxvLong) continue;
        const uint64_t nch = (d + kMxvChunk - 1) / kMxvChunk;
        const unsigned long long at = atomicAdd(count, (unsigned long long)nch);
        for (uint64_t i = 0; i < nch && at + i < cap; ++i) {
            cv[at + i] = (uint32_t)v;
            cs[at + i] = b + i * kMxvChunk;
        }
    }
}

// Build the graph's chunk list on first use (allocates; synchronises `st`).
template <typename E>
int ensure_plan(khop_graph *g, cudaStream_t st) {
    if (g->mxv_ready) return KHOP_OK;
    // each long list has more than kMxvLong edges (at most nnz / kMxvLong of
    // them) and adds at most one partial chunk to its nnz-share of whole ones
    const uint64_t cap = g->nnz / kMxvChunk + g->nnz / kMxvLong + 1;
    unsigned long long *cnt = &g->plain.ctl->pad[1];
    cudaError_t e = cudaMalloc(&g->mxv_cv, cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g->mxv_cs, cap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        mxv_plan_kernel<E><<<g->num_sms * 4, 256, 0, st>>>((const E *)g->cp, g->n, g->mxv_cv, g->mxv_cs, cap, cnt);
        e = cudaGetLastError();
    }
    unsigned long long nch = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nch, cnt, sizeof(nch), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(g->mxv_cv);
        cudaFree(g->mxv_cs);
        g->mxv_cv = nullptr;
        g->mxv_cs = nullptr;
        return cuda_status(e);
    }
    g->mxv_nch = nch < cap ? nch : cap;
    g->device_bytes += cap * (sizeof(uint32_t) + sizeof(unsigned long long));
    g->mxv_ready = true;
    return KHOP_OK;
}

template <typename E, int SR>
int launch_sr(khop_graph *g, const uint64_t *x, const uint32_t *mask, int comp, uint64_t *y, cudaStream_t st) {
    const int blocks = g->num_sms * 8;
    mxv_kernel<E, SR><<<blocks, 256, 0, st>>>((const E *)g->cp, g->ri, (const unsigned long long *)x, mask,
                                              comp ? 1u : 0u, g->n, g->nw, (unsigned long long *)y,
                                              &g->plain.ctl->pad[0]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && g->mxv_nch) {
        const uint64_t cb = std::min<uint64_t>((g->mxv_nch + 7) / 8, (uint64_t)g->num_sms * 8);
        mxv_chunk_kernel<E, SR><<<(unsigned)cb, 256, 0, st>>>(
            (const E *)g->cp, g->ri, (const unsigned long long *)x, mask, comp ? 1u : 0u, g->mxv_cv, g->mxv_cs,
            g->mxv_nch, (unsigned long long *)y, &g->plain.ctl->pad[0]);
        e = cudaGetLastError();
    }
    return cuda_status(e);
}

template <typename E>
int launch_mxv(khop_graph *g, int sr, const uint64_t *x, const uint32_t *mask, int comp, uint64_t *y,
               cudaStream_t st) {
    switch (sr) {
        case KHOP_SR_OR_AND: return launch_sr<E, KHOP_SR_OR_AND>(g, x, mask, comp, y, st);
        case KHOP_SR_PLUS_TIMES: return launch_sr<E, KHOP_SR_PLUS_TIMES>(g, x, mask, comp, y, st);
        case KHOP_SR_MIN_SECOND: return launch_sr<E, KHOP_SR_MIN_SECOND>(g, x, mask, comp, y, st);
        default: return launch_sr<E, KHOP_SR_MAX_SECOND>(g, x, mask, comp, y, st);
    }
}

}  // namespace
}  // namespace khop

extern "C" int khop_mxv(khop_graph *g, int semiring, const uint64_t *x, const uint32_t *mask, int mask_complement,
                        uint64_t *y, void *stream) {
    using namespace khop;
    if (!g || !x || !y) return KHOP_EINVAL;
    if (semiring < KHOP_SR_OR_AND || semiring > KHOP_SR_MAX_SECOND) return KHOP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = order_after_previous(g, st);
    // the in-edges scanned, for khop_mxv_stats (the plain control block's spare word)
    if (rc == KHOP_OK)
        rc = g->ewidth == 4 ? ensure_plan<uint32_t>(g, st) : ensure_plan<unsigned long long>(g, st);
    if (rc == KHOP_OK) rc = cuda_status(cudaMemsetAsync(&g->plain.ctl->pad[0], 0, sizeof(unsigned long long), st));
    if (rc == KHOP_OK)
        rc = g->ewidth == 4 ? launch_mxv<uint32_t>(g, semiring, x, mask, mask_complement, y, st)
                            : launch_mxv<unsigned long long>(g, semiring, x, mask, mask_complement, y, st);
    if (rc == KHOP_OK) rc = mark_done(g, st);
    return rc;
}

extern "C" int khop_mxv_stats(khop_graph *g, uint64_t *scanned) {
    using namespace khop;
    if (!g || !scanned) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    unsigned long long v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, &g->plain.ctl->pad[0], sizeof(v), cudaMemcpyDeviceToHost);
    *scanned = v;
    return cuda_status(e);
}
