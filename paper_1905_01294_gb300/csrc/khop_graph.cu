// Graph ingest (CSR upload, on-device CSC = A^T derivation, validation),
// tuning, sticky errors and the small C ABI helpers of libkhop.
#include <cstring>
#include <new>
#include <algorithm>

#include <vector>

#include "khop_internal.cuh"

using namespace khop;

namespace {

constexpr int kScanBlock = 1024;                 // threads of the scan kernels
constexpr int kScanTile = 2 * kScanBlock;        // elements per scan block

int bitlen(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

// ---- validation of the caller's CSR (raw input width W) --------------------
template <typename W>
__global__ void validate_kernel(const W *rp, const uint32_t *ci, uint64_t n, uint64_t nnz,
                                unsigned *bad) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = tid; i <= n; i += stride) {
        const uint64_t a = rp[i];
        if (i == 0 && a != 0) atomicOr(bad, 1u);
        if (i == n && a != nnz) atomicOr(bad, 2u);
        if (i < n && a > (uint64_t)rp[i + 1]) atomicOr(bad, 4u);
    }
    for (uint64_t e = tid; e < nnz; e += stride)
        if (ci[e] >= n) atomicOr(bad, 8u);
}

template <typename W, typename E>
__global__ void convert_kernel(const W *in, E *out, uint64_t count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = (E)in[i];
}

// ---- CSC derivation: in-degree histogram -> exclusive scan -> scatter -------
template <typename E>
__global__ void indegree_kernel(const uint32_t *ci, uint64_t nnz, E *cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd(&cnt[ci[e]], (E)1);
}

// Exclusive scan of one tile of kScanTile elements per block (in place);
// writes the tile total to sums[blockIdx.x].
template <typename E>
__global__ void __launch_bounds__(kScanBlock) scan_tile_kernel(E *x, uint64_t count, E *sums) {
    __shared__ E wsum[kScanBlock / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    const int t = threadIdx.x;
    const uint64_t i0 = base + 2 * t, i1 = i0 + 1;
    E a = i0 < count ? x[i0] : (E)0;
    E b = i1 < count ? x[i1] : (E)0;
    E pair = a + b;
    E incl = warp_inclusive_sum(pair);
    const int lane = t & 31, w = t >> 5;
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        E v = lane < kScanBlock / 32 ? wsum[lane] : (E)0;
        E vi = warp_inclusive_sum(v);
        if (lane < kScanBlock / 32) wsum[lane] = vi - v;
    }
    __syncthreads();
    const E excl = incl - pair + wsum[w];
    if (i0 < count) x[i0] = excl;
    if (i1 < count) x[i1] = excl + a;
    if (t == kScanBlock - 1) sums[blockIdx.x] = excl + pair;
}

template <typename E>
__global__ void scan_add_kernel(E *x, uint64_t count, const E *offs) {
    const uint64_t i = (uint64_t)blockIdx.x * kScanTile + threadIdx.x;
    const E o = offs[blockIdx.x];
    if (i < count) x[i] += o;
    if (i + kScanBlock < count) x[i + kScanBlock] += o;
}

// In-place exclusive scan of x[0..count) on the device (recursive over tiles).
template <typename E>
cudaError_t exclusive_scan(E *x, uint64_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const uint64_t tiles = (count + kScanTile - 1) / kScanTile;
    E *sums = nullptr;
    cudaError_t e = cudaMalloc(&sums, (tiles + 1) * sizeof(E));
    if (e != cudaSuccess) return e;
    scan_tile_kernel<E><<<(unsigned)tiles, kScanBlock, 0, st>>>(x, count, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess && tiles > 1) {
        e = exclusive_scan(sums, tiles, st);
        if (e == cudaSuccess) {
            scan_add_kernel<E><<<(unsigned)tiles, kScanBlock, 0, st>>>(x, count, sums);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(sums);
    return e != cudaSuccess ? e : e2;
}

// One warp per CSR row u: each edge u -> w is appended to column w of the CSC.
template <typename E>
__global__ void csc_scatter_kernel(const E *rp, const uint32_t *ci, uint64_t n, E *cursor,
                                   uint32_t *ri) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < n; u += nwarps) {
        const E b = rp[u], e = rp[u + 1];
        for (E p = b + lane; p < e; p += 32) {
            const uint32_t w = ci[p];
            const E pos = atomicAdd(&cursor[w], (E)1);
            ri[pos] = (uint32_t)u;
        }
    }
}

// In-list order.  A pull round stops at the first in-neighbour in the
// frontier, and high-degree vertices join the frontier early, so every in-list
// of at most kSortMax entries is sorted by the in-neighbour's out-degree,
// highest first (ties by id).  Each entry gets a 64-bit key -- inverted
// degree above, id below -- in a temporary array; one thread shell-sorts one
// list's keys; the ids are written back.  Longer lists keep their order.  No
// count depends on the order; it only shortens pull scans.
constexpr uint64_t kSortMax = 2048;

template <typename E>
__global__ void inlist_keys_kernel(const E *rp, const uint32_t *ri, uint64_t m,
                                   unsigned long long *key) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t u = ri[e];
        const uint64_t d = (uint64_t)(rp[u + 1] - rp[u]);
        const uint64_t inv = 0xffffffffull - (d < 0xffffffffull ? d : 0xffffffffull);
        key[e] = (inv << 32) | u;
    }
}

template <typename E>
__global__ void inlist_sort_kernel(const E *cp, unsigned long long *key, uint32_t *ri, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint64_t b = cp[v], d = (uint64_t)cp[v + 1] - b;
        if (d < 2 || d > kSortMax) continue;
        unsigned long long *x = key + b;
        for (uint64_t gap = d / 2; gap > 0; gap = gap == 2 ? 1 : gap * 5 / 11) {
            for (uint64_t i = gap; i < d; ++i) {
                const unsigned long long t = x[i];
                uint64_t j = i;
                while (j >= gap && x[j - gap] > t) { x[j] = x[j - gap]; j -= gap; }
                x[j] = t;
            }
        }
        for (uint64_t i = 0; i < d; ++i) ri[b + i] = (uint32_t)x[i];
    }
}

// Sort the in-lists (CSC columns; for a symmetric graph, the CSR rows).
template <typename E>
cudaError_t order_inlists(khop_graph *g, const E *cp, uint32_t *ri, cudaStream_t st) {
    if (g->nnz == 0) return cudaSuccess;
    unsigned long long *key = nullptr;
    cudaError_t e = cudaMalloc(&key, g->nnz * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    const int blocks = g->num_sms * 8;
    inlist_keys_kernel<E><<<blocks, 256, 0, st>>>((const E *)g->rp, ri, g->nnz, key);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        inlist_sort_kernel<E><<<blocks, 128, 0, st>>>(cp, key, ri, g->n);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(key);
    return e != cudaSuccess ? e : e2;
}

template <typename E>
cudaError_t build_csc(khop_graph *g, cudaStream_t st) {
    const uint64_t n = g->n, nnz = g->nnz;
    E *cp = nullptr, *cursor = nullptr;
    uint32_t *ri = nullptr;
    cudaError_t e = cudaMalloc(&cp, (n + 1) * sizeof(E));
    if (e == cudaSuccess) e = cudaMalloc(&ri, std::max<uint64_t>(nnz, 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&cursor, (n + 1) * sizeof(E));
    if (e != cudaSuccess) { cudaFree(cp); cudaFree(ri); cudaFree(cursor); return e; }
    g->cp = cp;
    g->ri = ri;
    g->device_bytes += (n + 1) * sizeof(E) + std::max<uint64_t>(nnz, 1) * sizeof(uint32_t);
    const int blocks = g->num_sms * 8;
    cudaMemsetAsync(cp, 0, (n + 1) * sizeof(E), st);
    if (nnz) indegree_kernel<E><<<blocks, 256, 0, st>>>(g->ci, nnz, cp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan(cp, n + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cursor, cp, (n + 1) * sizeof(E),
                                              cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && nnz) {
        csc_scatter_kernel<E><<<blocks, 256, 0, st>>>((const E *)g->rp, g->ci, n, cursor, ri);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(cursor);
    if (e == cudaSuccess && e2 == cudaSuccess) e = order_inlists<E>(g, cp, ri, st);
    return e != cudaSuccess ? e : e2;
}

// Bitmap of the vertices without in-edges (CSC column empty), and its count.
template <typename E>
__global__ void noin_kernel(const E *cp, uint64_t n, uint32_t nw, uint32_t *noin,
                            unsigned long long *count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw; i += stride) {
        uint32_t w = 0;
        for (int l = 0; l < 32; ++l) {
            const uint64_t v = (i << 5) + l;
            if (v < n && cp[v + 1] == cp[v]) w |= 1u << l;
        }
        noin[i] = w;
        if (w) atomicAdd(count, (unsigned long long)__popc(w));
    }
}

// Either-direction adjacency: row u of the result is out(u) followed by in(u).
// ro[u] = rp[u] + cp[u] (both are prefix sums).  One warp per vertex.
template <typename E, typename EO>
__global__ void union_rows_kernel(const E *rp, const uint32_t *ci, const E *cp, const uint32_t *ri,
                                  uint64_t n, EO *ro, uint32_t *co) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t u = warp; u <= n; u += nwarps) {
        const EO base = (EO)rp[u] + (EO)cp[u];
        if (lane == 0) ro[u] = base;
        if (u == n) break;
        const E o0 = rp[u], o1 = rp[u + 1], i0 = cp[u], i1 = cp[u + 1];
        for (E x = o0 + lane; x < o1; x += 32) co[(uint64_t)base + (x - o0)] = ci[x];
        const EO b2 = base + (EO)(o1 - o0);
        for (E x = i0 + lane; x < i1; x += 32) co[(uint64_t)b2 + (x - i0)] = ri[x];
    }
}

template <typename T>
cudaError_t dalloc(khop_graph *g, T **p, uint64_t count) {
    const size_t bytes = std::max<uint64_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) g->device_bytes += bytes;
    return e;
}

cudaError_t dalloc_raw(khop_graph *g, void **p, uint64_t bytes) {
    cudaError_t e = cudaMalloc(p, std::max<uint64_t>(bytes, 16));
    if (e == cudaSuccess) g->device_bytes += std::max<uint64_t>(bytes, 16);
    return e;
}

}  // namespace
namespace khop { void free_batch_state(BatchState &b); }
namespace {

void free_graph(khop_graph *g) {
    if (!g) return;
    if (g->cp && g->cp != g->rp) cudaFree(g->cp);
    if (g->ri && g->ri != g->ci) cudaFree(g->ri);
    cudaFree(g->rp);
    cudaFree(g->ci);
    cudaFree(g->noin);
    free_plain_state(g->plain);
    free_batch_state(g->batch);
    free_batch_state(g->batch2);
    free_batch_state(g->batch4);
    cudaFree(g->mxv_cv);
    cudaFree(g->mxv_cs);
    if (g->done) cudaEventDestroy(g->done);
    delete g;
}

}  // namespace

namespace khop {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return KHOP_OK;
    if (e == cudaErrorMemoryAllocation) return KHOP_ENOMEM;
    return KHOP_ECUDA;
}

// Order a call after the previous call on g when it comes on another stream.
// A stream being captured into a CUDA graph is left alone: its captured work
// runs when the graph is launched, and ordering the launches is the caller's.
int order_after_previous(khop_graph *g, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return KHOP_ECUDA;
    if (cs != cudaStreamCaptureStatusNone) return KHOP_OK;
    if (g->have_last && g->last_stream != s)
        return cuda_status(cudaStreamWaitEvent(s, g->done, 0));
    return KHOP_OK;
}

int mark_done(khop_graph *g, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return KHOP_ECUDA;
    if (cs != cudaStreamCaptureStatusNone) return KHOP_OK;
    cudaError_t e = cudaEventRecord(g->done, s);
    g->last_stream = s;
    g->have_last = true;
    return cuda_status(e);
}

namespace kcache {
// Per (kernel, device): the dynamic shared memory the kernel was opened to;
// per (kernel, device, block, smem): its resident CTAs per SM.
struct KernelAttr { const void *fn; int dev; size_t smem; };
struct KernelOcc { const void *fn; int dev; int block; size_t smem; int per_sm; };
static std::mutex g_kmu;
static std::vector<KernelAttr> g_kattr;
static std::vector<KernelOcc> g_kocc;
}  // namespace kcache

int launch_shape(const void *kernel, int block, size_t smem, int want_per_sm, int num_sms, int *grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = -1;
    {
        using namespace kcache;
        std::lock_guard<std::mutex> lk(g_kmu);
        KernelAttr *at = nullptr;
        for (KernelAttr &x : g_kattr)
            if (x.fn == kernel && x.dev == dev) at = &x;
        if (!at || at->smem < smem) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_status(e);
            if (at) at->smem = smem;
            else g_kattr.push_back(KernelAttr{kernel, dev, smem});
        }
        for (const KernelOcc &x : g_kocc)
            if (x.fn == kernel && x.dev == dev && x.block == block && x.smem == smem) per_sm = x.per_sm;
        if (per_sm < 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
            if (e != cudaSuccess) return cuda_status(e);
            g_kocc.push_back(KernelOcc{kernel, dev, block, smem, per_sm});
        }
    }
    if (per_sm <= 0) return KHOP_EINVAL;
    if (want_per_sm > 0) per_sm = std::min(per_sm, want_per_sm);
    *grid = per_sm * num_sms;
    return KHOP_OK;
}

int cooperative_grid(const void *kernel, int block, size_t smem, int want_per_sm, int num_sms,
                     int *grid) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm <= 0) return KHOP_EINVAL;
    if (want_per_sm > 0) per_sm = std::min(per_sm, want_per_sm);
    *grid = per_sm * num_sms;
    return KHOP_OK;
}

void free_batch_state(BatchState &b) {
    cudaFree(b.V);
    for (int i = 0; i < 3; ++i) cudaFree(b.F[i]);
    for (int i = 0; i < 2; ++i) { cudaFree(b.Q[i]); cudaFree(b.Qpre[i]); cudaFree(b.TF[i]); cudaFree(b.S[i]); }
    cudaFree(b.ctl);
    cudaFree(b.part);
    cudaFree(b.order);
    cudaFree(b.hv);
    cudaFree(b.hend);
    cudaFree(b.hneed);
    cudaFree(b.hacc);
    cudaFree(b.ch_item);
    cudaFree(b.ch_start);
    b = BatchState{};
}

void free_plain_state(PlainState &p) {
    cudaFree(p.V);
    cudaFree(p.V2);
    for (auto &f : p.F) cudaFree(f);
    for (int i = 0; i < 2; ++i) { cudaFree(p.Qpre[i]); cudaFree(p.Qrs[i]); cudaFree(p.TF[i]); }
    cudaFree(p.ctl);
    p = PlainState{};
}

// Allocate (and zero) a plain traversal state for graph g; synchronises.
int alloc_plain_state(khop_graph *g, PlainState &p) {
    const uint64_t n = g->n, nw = g->nw;
    const uint64_t before = g->device_bytes;
    p = PlainState{};
    cudaError_t e = dalloc(g, &p.V, nw);
    if (e == cudaSuccess) e = dalloc(g, &p.V2, nw);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(g, &p.F[i], nw);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc_raw(g, &p.Qpre[i], n * (uint64_t)g->ewidth);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc_raw(g, &p.Qrs[i], n * (uint64_t)g->ewidth);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc(g, &p.TF[i], g->tf_cap);
    if (e == cudaSuccess) e = dalloc(g, &p.ctl, 1);
    if (e == cudaSuccess) e = cudaMemset(p.V, 0, nw * 4);
    if (e == cudaSuccess) e = cudaMemset(p.V2, 0, nw * 4);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemset(p.F[i], 0, nw * 4);
    if (e == cudaSuccess) e = cudaMemset(p.ctl, 0, sizeof(CtlBlock));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plain_state(p);
        g->device_bytes = before;
        return cuda_status(e);
    }
    p.bytes = g->device_bytes - before;
    return KHOP_OK;
}

// Allocate a bit-sliced batch state for graph g (no device sync needed by
// the caller afterwards).  *bytes receives its size.
int alloc_batch_state(khop_graph *g, BatchState &b, uint64_t *bytes, int lw, bool sinks) {
    const uint64_t n = g->n;
    const uint64_t before = g->device_bytes;
    b = BatchState{};
    b.lw = lw;
    b.part_rows = (uint64_t)g->num_sms * 4;
    // a deferred in-list has more than 4096 edges left, so at most nnz / 4096
    // vertices defer per round, in at most 2 nnz / 4096 + 1 chunks of 4096
    b.hcap = std::min<uint64_t>(n, g->nnz / 4096 + 1);
    b.ccap = 2 * (g->nnz / 4096) + 2;
    cudaError_t e = dalloc(g, &b.V, n * lw);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(g, &b.F[i], n * lw);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc(g, &b.Q[i], n);
    for (int i = 0; i < 2 && e == cudaSuccess && sinks; ++i) e = dalloc(g, &b.S[i], n);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc_raw(g, &b.Qpre[i], n * g->ewidth);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc(g, &b.TF[i], g->tf_cap);
    if (e == cudaSuccess) e = dalloc(g, &b.ctl, 1);
    if (e == cudaSuccess) e = dalloc(g, &b.part, 2 * b.part_rows * 64 * lw);
    if (e == cudaSuccess) e = dalloc(g, &b.hv, b.hcap);
    if (e == cudaSuccess) e = dalloc_raw(g, &b.hend, b.hcap * g->ewidth);
    if (e == cudaSuccess) e = dalloc(g, &b.hneed, b.hcap * lw);
    if (e == cudaSuccess) e = dalloc(g, &b.hacc, b.hcap * lw);
    if (e == cudaSuccess) e = dalloc(g, &b.ch_item, b.ccap);
    if (e == cudaSuccess) e = dalloc_raw(g, &b.ch_start, b.ccap * g->ewidth);
    if (e == cudaSuccess) e = cudaMemset(b.hacc, 0, b.hcap * lw * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b.part, 0, 2 * b.part_rows * 64 * lw * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b.V, 0, n * lw * sizeof(uint64_t));
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemset(b.F[i], 0, n * lw * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMemset(b.ctl, 0, sizeof(CtlBlock));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_batch_state(b);
        g->device_bytes = before;
        return cuda_status(e);
    }
    b.bytes = g->device_bytes - before;
    if (bytes) *bytes = b.bytes;
    return KHOP_OK;
}

// Bytes a batch state of graph g takes (for admission decisions).
uint64_t batch_state_bytes(const khop_graph *g) {
    const uint64_t n = g->n, W = (uint64_t)g->ewidth;
    const uint64_t hcap = std::min<uint64_t>(n, g->nnz / 4096 + 1), ccap = 2 * (g->nnz / 4096) + 2;
    return 4 * n * 8 + 2 * n * 4 + 2 * n * W + 2 * g->tf_cap * 4 + sizeof(CtlBlock) +
           2 * (uint64_t)g->num_sms * 4 * 64 * 8 + hcap * (4 + W + 16) + ccap * (4 + W);
}

uint64_t plain_state_bytes(const khop_graph *g) {
    return 5ull * g->nw * 4 + 4 * g->n * (uint64_t)g->ewidth + 2 * g->tf_cap * 4 + sizeof(CtlBlock);
}

int ensure_batch_state(khop_graph *g, int lw) {
    BatchState &b = lw == 4 ? g->batch4 : (lw == 2 ? g->batch2 : g->batch);
    if (b.V) return KHOP_OK;
    return alloc_batch_state(g, b, nullptr, lw);
}

}  // namespace khop

// ===========================================================================
// C ABI

extern "C" {

const char *khop_strerror(int status) {
    switch (status) {
        case KHOP_OK: return "success";
        case KHOP_EINVAL: return "invalid argument";
        case KHOP_ENOMEM: return "out of memory";
        case KHOP_ECUDA: return "CUDA runtime error";
        case KHOP_EBUSY: return "busy: admission refused";
        case KHOP_ETIMEDOUT: return "timed out";
        case KHOP_ESHUTDOWN: return "server shutting down";
        case KHOP_EDEVICE: return "device-side error recorded";
        default: return "unknown status";
    }
}

int khop_version(void) { return KHOP_VERSION_NUM; }

int khop_graph_create(uint64_t n, const void *row_ptr, int row_ptr_bytes, const uint32_t *col_idx,
                      uint64_t nnz, uint32_t flags, void *stream, khop_graph **out) {
    if (!out) return KHOP_EINVAL;
    *out = nullptr;
    if (n == 0 || n >= (1ull << 32) || !row_ptr || (nnz && !col_idx)) return KHOP_EINVAL;
    if (row_ptr_bytes != 4 && row_ptr_bytes != 8) return KHOP_EINVAL;
    if (row_ptr_bytes == 4 && nnz >= (1ull << 32)) return KHOP_EINVAL;
    if (flags & ~(uint32_t)(KHOP_DEVICE_PTRS | KHOP_SYMMETRIC | KHOP_VALIDATE | KHOP_WIDE_OFFSETS |
                            KHOP_REVERSE | KHOP_UNDIRECTED))
        return KHOP_EINVAL;
    if (bitlen(n) + bitlen(nnz) > 64) return KHOP_EINVAL;
    const bool undirected = (flags & KHOP_UNDIRECTED) && !(flags & KHOP_SYMMETRIC);
    const bool reverse = (flags & KHOP_REVERSE) && !(flags & (KHOP_SYMMETRIC | KHOP_UNDIRECTED));
    if (undirected && bitlen(n) + bitlen(2 * nnz) > 64) return KHOP_EINVAL;
    const bool on_device = flags & KHOP_DEVICE_PTRS;
    cudaStream_t st = (cudaStream_t)stream;

    khop_graph *g = new (std::nothrow) khop_graph();
    if (!g) return KHOP_ENOMEM;
    g->n = n;
    g->nnz = nnz;
    g->ewidth = (nnz < (1ull << 32) && !(flags & KHOP_WIDE_OFFSETS)) ? 4 : 8;
    g->symmetric = flags & KHOP_SYMMETRIC;
    g->nw = (uint32_t)((n + 31) / 32);
    g->ebits = (uint32_t)(64 - bitlen(n));
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }

    // Raw input on the device (copied from the host if needed).
    void *raw_rp = nullptr;
    uint32_t *raw_ci = nullptr;
    bool own_raw = false;
    if (on_device) {
        raw_rp = const_cast<void *>(row_ptr);
        raw_ci = const_cast<uint32_t *>(col_idx);
    } else {
        own_raw = true;
        e = cudaMalloc(&raw_rp, (n + 1) * row_ptr_bytes);
        if (e == cudaSuccess && nnz) e = cudaMalloc(&raw_ci, nnz * sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(raw_rp, row_ptr, (n + 1) * row_ptr_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && nnz)
            e = cudaMemcpyAsync(raw_ci, col_idx, nnz * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    }
    auto cleanup_raw = [&]() {
        if (own_raw) { cudaFree(raw_rp); cudaFree(raw_ci); }
    };
    if (e != cudaSuccess) { cudaStreamSynchronize(st); cleanup_raw(); free_graph(g); return cuda_status(e); }

    const int blocks = g->num_sms * 8;
    if (flags & KHOP_VALIDATE) {
        unsigned *bad = nullptr;
        unsigned hbad = 0;
        e = cudaMalloc(&bad, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) {
            if (row_ptr_bytes == 4)
                validate_kernel<uint32_t><<<blocks, 256, 0, st>>>((const uint32_t *)raw_rp, raw_ci, n, nnz, bad);
            else
                validate_kernel<uint64_t><<<blocks, 256, 0, st>>>((const uint64_t *)raw_rp, raw_ci, n, nnz, bad);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(bad);
        if (e != cudaSuccess) { cleanup_raw(); free_graph(g); return cuda_status(e); }
        if (hbad) { cleanup_raw(); free_graph(g); return KHOP_EINVAL; }
    }

    // Internal CSR with edge offsets of g->ewidth bytes.
    e = dalloc_raw(g, &g->rp, (n + 1) * (uint64_t)g->ewidth);
    if (e == cudaSuccess) e = dalloc(g, &g->ci, nnz);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(g->ci, raw_ci, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        if (row_ptr_bytes == 4 && g->ewidth == 4)
            e = cudaMemcpyAsync(g->rp, raw_rp, (n + 1) * 4, cudaMemcpyDeviceToDevice, st);
        else if (row_ptr_bytes == 8 && g->ewidth == 8)
            e = cudaMemcpyAsync(g->rp, raw_rp, (n + 1) * 8, cudaMemcpyDeviceToDevice, st);
        else if (row_ptr_bytes == 8)
            convert_kernel<uint64_t, uint32_t><<<blocks, 256, 0, st>>>((const uint64_t *)raw_rp, (uint32_t *)g->rp, n + 1);
        else
            convert_kernel<uint32_t, uint64_t><<<blocks, 256, 0, st>>>((const uint32_t *)raw_rp, (uint64_t *)g->rp, n + 1);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup_raw();
    if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }

    // CSC (in-edges).  A symmetric graph is its own transpose.
    if (g->symmetric) {
        g->cp = g->rp;
        g->ri = g->ci;
        e = g->ewidth == 4 ? order_inlists<uint32_t>(g, (const uint32_t *)g->rp, g->ci, st)
                           : order_inlists<unsigned long long>(g, (const unsigned long long *)g->rp, g->ci, st);
        if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }
    } else {
        e = g->ewidth == 4 ? build_csc<uint32_t>(g, st) : build_csc<unsigned long long>(g, st);
        if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }
        if (undirected) {
            // A OR A^T: each row is the out-list then the in-list; the result is
            // its own transpose.
            const uint64_t nnz2 = 2 * nnz;
            const int ew2 = (nnz2 < (1ull << 32) && !(flags & KHOP_WIDE_OFFSETS)) ? 4 : 8;
            void *ro = nullptr;
            uint32_t *co = nullptr;
            e = dalloc_raw(g, &ro, (n + 1) * (uint64_t)ew2);
            if (e == cudaSuccess) e = dalloc(g, &co, nnz2);
            if (e == cudaSuccess) {
                if (g->ewidth == 4 && ew2 == 4)
                    union_rows_kernel<uint32_t, uint32_t><<<blocks, 256, 0, st>>>(
                        (const uint32_t *)g->rp, g->ci, (const uint32_t *)g->cp, g->ri, n, (uint32_t *)ro, co);
                else if (g->ewidth == 4)
                    union_rows_kernel<uint32_t, unsigned long long><<<blocks, 256, 0, st>>>(
                        (const uint32_t *)g->rp, g->ci, (const uint32_t *)g->cp, g->ri, n,
                        (unsigned long long *)ro, co);
                else
                    union_rows_kernel<unsigned long long, unsigned long long><<<blocks, 256, 0, st>>>(
                        (const unsigned long long *)g->rp, g->ci, (const unsigned long long *)g->cp, g->ri, n,
                        (unsigned long long *)ro, co);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { cudaFree(ro); cudaFree(co); free_graph(g); return cuda_status(e); }
            const uint64_t W = (uint64_t)g->ewidth;
            cudaFree(g->rp);
            cudaFree(g->ci);
            cudaFree(g->cp);
            cudaFree(g->ri);
            g->device_bytes -= 2 * ((n + 1) * W + std::max<uint64_t>(nnz, 1) * sizeof(uint32_t));
            g->rp = ro;
            g->ci = co;
            g->cp = ro;
            g->ri = co;
            g->nnz = nnz2;
            g->ewidth = ew2;
            g->ebits = (uint32_t)(64 - bitlen(n));
            g->symmetric = true;
            e = g->ewidth == 4 ? order_inlists<uint32_t>(g, (const uint32_t *)g->rp, g->ci, st)
                               : order_inlists<unsigned long long>(g, (const unsigned long long *)g->rp, g->ci, st);
            if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }
        } else if (reverse) {
            // in-neighbourhoods: traverse the transpose; its own transpose is A
            std::swap(g->rp, g->cp);
            std::swap(g->ci, g->ri);
            e = g->ewidth == 4 ? order_inlists<uint32_t>(g, (const uint32_t *)g->cp, g->ri, st)
                               : order_inlists<unsigned long long>(g, (const unsigned long long *)g->cp, g->ri, st);
            if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }
        }
    }

    // Plain traversal state and the in-edge-less vertex map.
    g->tf_cap = g->nnz / 256 + 2;
    const uint64_t nw = g->nw;
    e = dalloc(g, &g->noin, nw);
    if (e == cudaSuccess) {
        unsigned long long *cnt = nullptr;
        e = cudaMalloc(&cnt, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) {
            if (g->ewidth == 4)
                noin_kernel<uint32_t><<<blocks, 256, 0, st>>>((const uint32_t *)g->cp, n, g->nw, g->noin, cnt);
            else
                noin_kernel<unsigned long long><<<blocks, 256, 0, st>>>((const unsigned long long *)g->cp, n, g->nw, g->noin, cnt);
            e = cudaGetLastError();
        }
        unsigned long long h = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        g->n_noin = h;
        cudaFree(cnt);
    }
    if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }
    int prc = alloc_plain_state(g, g->plain);
    if (prc != KHOP_OK) { free_graph(g); return prc; }
    e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
    if (e != cudaSuccess) { free_graph(g); return cuda_status(e); }

    g->tune.direction = KHOP_DIR_AUTO;
    g->tune.alpha = 14.0f;
    g->tune.beta = 24.0f;
    g->tune.block_threads = 512;
    g->tune.blocks_per_sm = 2;
    g->tune.push_tile = 2048;
    g->tune.batch_alpha = 14.0f;
    g->tune.batch_beta = 24.0f;
    g->tune.batch_push_tile = 2048;
    *out = g;
    return KHOP_OK;
}

int khop_graph_destroy(khop_graph *g) {
    if (!g) return KHOP_EINVAL;
    cudaDeviceSynchronize();
    free_graph(g);
    return KHOP_OK;
}

int khop_graph_info(const khop_graph *g, uint64_t *n, uint64_t *nnz) {
    if (!g) return KHOP_EINVAL;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return KHOP_OK;
}

int khop_graph_device_bytes(const khop_graph *g, uint64_t *bytes) {
    if (!g || !bytes) return KHOP_EINVAL;
    *bytes = g->device_bytes;
    return KHOP_OK;
}

int khop_graph_get_tuning(const khop_graph *g, khop_tuning *t) {
    if (!g || !t) return KHOP_EINVAL;
    *t = g->tune;
    return KHOP_OK;
}

int khop_graph_set_tuning(khop_graph *g, const khop_tuning *t) {
    if (!g || !t) return KHOP_EINVAL;
    if (t->direction < 0 || t->direction > KHOP_DIR_PULL) return KHOP_EINVAL;
    if (t->alpha < 0 || t->beta < 0 || t->batch_alpha < 0 || t->batch_beta < 0) return KHOP_EINVAL;
    if (t->block_threads && t->block_threads != 256 && t->block_threads != 512 &&
        t->block_threads != 1024)
        return KHOP_EINVAL;
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 8) return KHOP_EINVAL;
    if (t->push_tile && (t->push_tile < 256 || t->push_tile > 8192 ||
                         (t->push_tile & (t->push_tile - 1))))
        return KHOP_EINVAL;
    if (t->batch_push_tile && (t->batch_push_tile < 256 || t->batch_push_tile > 8192 ||
                               (t->batch_push_tile & (t->batch_push_tile - 1))))
        return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    g->tune.direction = t->direction;
    if (t->alpha > 0) g->tune.alpha = t->alpha;
    if (t->beta > 0) g->tune.beta = t->beta;
    if (t->block_threads) g->tune.block_threads = t->block_threads;
    if (t->blocks_per_sm) g->tune.blocks_per_sm = t->blocks_per_sm;
    if (t->push_tile) g->tune.push_tile = t->push_tile;
    if (t->batch_alpha > 0) g->tune.batch_alpha = t->batch_alpha;
    if (t->batch_beta > 0) g->tune.batch_beta = t->batch_beta;
    if (t->batch_push_tile) g->tune.batch_push_tile = t->batch_push_tile;
    return KHOP_OK;
}

int khop_get_error(khop_graph *g, uint32_t *bits) {
    if (!g || !bits) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    unsigned a = 0, b = 0;
    e = cudaMemcpy(&a, &g->plain.ctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && g->batch.ctl)
        e = cudaMemcpy(&b, &g->batch.ctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    for (BatchState *w : {&g->batch2, &g->batch4})
        if (e == cudaSuccess && w->ctl) {
            unsigned bw = 0;
            e = cudaMemcpy(&bw, &w->ctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
            b |= bw;
        }
    if (e == cudaSuccess) e = cudaMemset(&g->plain.ctl->err, 0, sizeof(unsigned));
    if (e == cudaSuccess && g->batch.ctl) e = cudaMemset(&g->batch.ctl->err, 0, sizeof(unsigned));
    if (e == cudaSuccess && g->batch2.ctl) e = cudaMemset(&g->batch2.ctl->err, 0, sizeof(unsigned));
    if (e == cudaSuccess && g->batch4.ctl) e = cudaMemset(&g->batch4.ctl->err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    *bits = a | b;
    return cuda_status(e);
}

int khop_graph_set_wait_limit(khop_graph *g, uint64_t timeout_ns) {
    if (!g || timeout_ns > 60000000000ull) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    g->timeout_ns = timeout_ns ? timeout_ns : 2000000000ull;
    return KHOP_OK;
}

int khop_graph_test_absent_cta(khop_graph *g, uint32_t barrier_index) {
    if (!g) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    g->absent_at = barrier_index;
    return KHOP_OK;
}

}  // extern "C"
