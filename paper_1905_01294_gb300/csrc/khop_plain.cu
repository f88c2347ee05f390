// Plain single-query k-hop count.
//
// One cooperative, persistent launch runs a list of queries one after another.
// A query is the masked (OR, AND) frontier iteration
//     q_r = (A^T q_{r-1}) AND NOT v_{r-1},   v_r = v_{r-1} OR q_r,   r = 1..k
// and its count is sum_r |q_r| = popcount(v_k) - 1.  Each round is one of:
//   push  (SpMSpV): the frontier is a queue of vertices with their out-edge
//         prefix; the frontier's out-edges are cut into fixed tiles of T edges
//         (merge-path over the frontier degrees: the tile -> first-item map is
//         written when the queue is built), and each edge u -> w does a
//         test-and-set of w's visited bit;
//   pull  (masked SpMV): every unvisited vertex scans its in-edges (CSC) for
//         a parent in the frontier bitmap and stops at the first one found.
// The direction follows Beamer's switch; the vertex counts come from
// warp ballots/popcounts.  Rounds are separated by a software grid barrier.
#include <algorithm>
#include <cmath>

#include "khop_internal.cuh"

namespace khop {
namespace {

enum { DIR_PUSH = 0, DIR_PULL = 1 };

constexpr int kPushUnroll = 4;   // edges in flight per thread in a push tile
constexpr int kLaneScan = 4;     // in-edges a lane scans alone before the warp helps

template <typename E>
struct PlainArgs {
    uint64_t n, nnz;
    uint32_t nw;
    int symmetric;
    const E *rp;             // CSR row offsets [n+1]
    const uint32_t *ci;      // CSR heads [nnz]
    const E *cp;             // CSC column offsets [n+1]
    const uint32_t *ri;      // CSC tails [nnz]
    uint32_t *V;             // visited bitmap [nw]
    uint32_t *F0, *F1, *F2;  // frontier bitmaps [nw], rotating per round
    E *Qpre0, *Qpre1;        // queue: out-edge prefix per item [n], double-buffered
    E *Qrs0, *Qrs1;          // queue: row start per item [n]
    uint32_t *TF0, *TF1;     // first queue item of each push tile
    CtlBlock *ctl;
    const uint32_t *seeds;
    const uint32_t *ks;      // per-query k, or null (then k_all)
    uint32_t k_all;
    uint64_t nq;
    uint64_t *out;
    uint64_t *out_te;
    khop_query_stats *stats;
    uint64_t *per_hop;
    uint32_t hop_stride;
    int direction;
    float alpha, beta;
    uint32_t tile_log2;
    uint32_t ebits;
    uint64_t pull_cap;       // queue items a pull round writes (enough for a switch back to push)
    uint64_t timeout_ns;
};

template <typename T>
__device__ __forceinline__ T sel3(T x0, T x1, T x2, unsigned i) {
    return i == 0 ? x0 : (i == 1 ? x1 : x2);
}

template <typename E>
struct Round {
    bool first, last;
    uint32_t seed;
    const uint32_t *Fin;
    uint32_t *Fout;
    const E *Qpre_in, *Qrs_in;
    const uint32_t *TF_in;
    E *Qpre_out, *Qrs_out;
    uint32_t *TF_out;
    unsigned long long *qpack_out;
    uint64_t cap;            // queue items this round may write
    uint64_t items_in, mf;   // input frontier: queue items, out-edges
};

// Warp-collective bookkeeping of newly visited vertices.  `disc` marks a
// lane's new vertex w with row start rs and out-degree d.  The count goes to
// the CTA counter.  Unless this is the last round, vertices with out-edges
// are appended to the next queue with their out-edge prefix (one packed
// 64-bit atomic per warp gives both the slot and the prefix), and every push
// tile that begins inside such a row records the row's slot.  set_f marks the
// vertex in the next frontier bitmap (push rounds; pull rounds store whole
// words).  Only vertices with out-edges need the bit: a pull round looks for
// parents, and a parent has an out-edge.
template <typename E>
__device__ __forceinline__ void record(const PlainArgs<E> &a, const Round<E> &R, bool disc,
                                       uint32_t w, E rs, E d, bool set_f,
                                       unsigned long long *s_cnt) {
    const unsigned m = __ballot_sync(FULL, disc);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    if (lane == 0) atomicAdd(s_cnt, (unsigned long long)__popc(m));
    if (R.last) return;
    const bool has = disc && d > 0;
    if (has && set_f) atomicOr(&R.Fout[w >> 5], 1u << (w & 31));
    const unsigned hm = __ballot_sync(FULL, has);
    if (hm == 0u) return;
    const E dd = has ? d : (E)0;
    const E incl = warp_inclusive_sum(dd);
    const E tot = __shfl_sync(FULL, incl, 31);
    const int leader = __ffs(hm) - 1;
    unsigned long long old = 0;
    if (lane == leader)
        old = atomicAdd(R.qpack_out,
                        ((unsigned long long)__popc(hm) << a.ebits) + (unsigned long long)tot);
    old = __shfl_sync(FULL, old, leader);
    if (has) {
        const uint64_t pos = (old >> a.ebits) + (uint64_t)__popc(hm & lanemask_lt());
        const uint64_t pre = (old & ((1ull << a.ebits) - 1ull)) + (uint64_t)(incl - dd);
        if (pos < R.cap) {
            R.Qpre_out[pos] = (E)pre;
            R.Qrs_out[pos] = rs;
            const uint64_t jf = (pre + (1ull << a.tile_log2) - 1ull) >> a.tile_log2;
            const uint64_t jl = (pre + (uint64_t)d - 1ull) >> a.tile_log2;
            for (uint64_t j = jf; j <= jl; ++j) R.TF_out[j] = (uint32_t)pos;
        }
    }
}

// Push round: tiles of T consecutive frontier out-edges, one CTA per tile.
template <typename E, int BLOCK>
__device__ __forceinline__ void push_round(const PlainArgs<E> &a, const Round<E> &R, E *s_pre, E *s_rs,
                           unsigned long long *s_cnt) {
    const uint32_t tl = a.tile_log2;
    const uint64_t T = 1ull << tl;
    const uint64_t ntiles = (R.mf + T - 1) >> tl;
    for (uint64_t j = blockIdx.x; j < ntiles; j += gridDim.x) {
        const uint64_t e0 = j << tl;
        const uint64_t e1 = min(e0 + T, R.mf);
        uint32_t nitems;
        if (R.first) {
            if (threadIdx.x == 0) {
                s_pre[0] = (E)0;
                s_rs[0] = a.rp[R.seed];
            }
            nitems = 1;
        } else {
            const uint64_t i0 = R.TF_in[j];
            const uint64_t il = (j + 1 < ntiles) ? (uint64_t)R.TF_in[j + 1] : R.items_in - 1;
            nitems = (uint32_t)(il - i0 + 1);
            for (uint32_t t = threadIdx.x; t < nitems; t += BLOCK) {
                s_pre[t] = R.Qpre_in[i0 + t];
                s_rs[t] = R.Qrs_in[i0 + t];
            }
        }
        __syncthreads();
        uint32_t hint = 0;
        for (uint64_t base = e0; base < e1; base += (uint64_t)BLOCK * kPushUnroll) {
            uint32_t w[kPushUnroll];
            bool ok[kPushUnroll];
#pragma unroll
            for (int u = 0; u < kPushUnroll; ++u) {
                const uint64_t e = base + (uint64_t)u * BLOCK + threadIdx.x;
                ok[u] = e < e1;
                w[u] = 0;
                if (ok[u]) {
                    uint32_t lo = hint, hi = nitems - 1;   // largest item with prefix <= e
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if ((uint64_t)s_pre[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    hint = lo;
                    w[u] = a.ci[(uint64_t)s_rs[lo] + (e - (uint64_t)s_pre[lo])];
                }
            }
#pragma unroll
            for (int u = 0; u < kPushUnroll; ++u) {
                bool disc = false;
                if (ok[u]) {
                    const uint32_t wi = w[u] >> 5, bit = 1u << (w[u] & 31);
                    if (!(a.V[wi] & bit)) disc = !(atomicOr(&a.V[wi], bit) & bit);
                }
                E rs = 0, d = 0;
                if (disc && !R.last) {
                    rs = a.rp[w[u]];
                    d = a.rp[w[u] + 1] - rs;
                }
                record(a, R, disc, w[u], rs, d, true, s_cnt);
            }
        }
        __syncthreads();
    }
}

// Pull round: one warp per 32-vertex bitmap word; each unvisited vertex looks
// for an in-neighbour in the frontier bitmap and stops at the first.
template <typename E, int BLOCK>
__device__ __forceinline__ void pull_round(const PlainArgs<E> &a, const Round<E> &R, unsigned long long *s_cnt,
                           unsigned long long *s_scan) {
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * BLOCK) >> 5;
    uint64_t scanned = 0;
    for (uint64_t i = gwarp; i < a.nw; i += nwarps) {
        const uint32_t Vw = a.V[i];
        const uint64_t v = (i << 5) + (uint64_t)lane;
        const bool unv = v < a.n && !((Vw >> lane) & 1u);
        if (__ballot_sync(FULL, unv) == 0u) {
            if (lane == 0) R.Fout[i] = 0u;
            continue;
        }
        E b = 0, e = 0;
        if (unv) {
            b = a.cp[v];
            e = a.cp[v + 1];
        }
        bool found = false;
        E pos = b;
        for (int t = 0; t < kLaneScan; t += 2) {
            const bool l0 = unv && !found && pos < e;
            const bool l1 = l0 && pos + 1 < e;
            uint32_t u0 = 0, u1 = 0;
            if (l0) u0 = a.ri[pos];
            if (l1) u1 = a.ri[pos + 1];
            bool h = false;
            if (l0) h = (R.Fin[u0 >> 5] >> (u0 & 31)) & 1u;
            if (l1) h = h || ((R.Fin[u1 >> 5] >> (u1 & 31)) & 1u);
            scanned += (uint64_t)l0 + (uint64_t)l1;
            pos += (E)l0 + (E)l1;
            found = found || h;
            if (!__any_sync(FULL, unv && !found && pos < e)) break;
        }
        unsigned rem = __ballot_sync(FULL, unv && !found && pos < e);
        while (rem) {
            const int L = __ffs(rem) - 1;
            const E lb = __shfl_sync(FULL, pos, L), le = __shfl_sync(FULL, e, L);
            bool hit = false;
            for (E c = lb; c < le; c += 32) {
                const E idx = c + (E)lane;
                bool h = false;
                if (idx < le) {
                    const uint32_t u = a.ri[idx];
                    h = (R.Fin[u >> 5] >> (u & 31)) & 1u;
                    ++scanned;
                }
                if (__any_sync(FULL, h)) { hit = true; break; }
            }
            if (lane == L) found = hit;
            rem &= rem - 1u;
        }
        const unsigned nm = __ballot_sync(FULL, found);
        if (lane == 0) {
            R.Fout[i] = nm;
            if (nm) a.V[i] = Vw | nm;
        }
        E rs = 0, d = 0;
        if (found && !R.last) {
            if (a.symmetric) { rs = b; d = e - b; }
            else { rs = a.rp[v]; d = a.rp[v + 1] - rs; }
        }
        record(a, R, found, (uint32_t)v, rs, d, false, s_cnt);
    }
    scanned = warp_sum(scanned);
    if (lane == 0 && scanned) atomicAdd(s_scan, (unsigned long long)scanned);
}

// Answer queries that need no traversal (k = 0, or a seed >= n) and return
// the index of the next query that does.  Only thread 0 of CTA 0 writes.
template <typename E>
__device__ __forceinline__ uint64_t skip_trivial(const PlainArgs<E> &a, uint64_t q, bool b0,
                                                 uint64_t &t_prev) {
    for (; q < a.nq; ++q) {
        const uint32_t s = a.seeds[q];
        const uint32_t k = a.ks ? a.ks[q] : a.k_all;
        if (s < a.n && k > 0) break;
        if (b0) {
            const bool bad = s >= a.n;
            const uint64_t now = globaltimer_ns();
            a.out[q] = bad ? ~0ull : 0ull;
            if (a.out_te) a.out_te[q] = bad ? ~0ull : 0ull;
            if (a.stats) {
                khop_query_stats st{t_prev, now, bad ? ~0ull : 0ull, 0ull, 0u, 0u};
                a.stats[q] = st;
            }
            if (a.per_hop)
                for (uint32_t r = 0; r < a.hop_stride; ++r)
                    a.per_hop[q * a.hop_stride + r] = (r == 0 && !bad) ? 1ull : 0ull;
            if (bad) atomicOr(&a.ctl->err, (unsigned)KHOP_DEVERR_SEED);
            t_prev = now;
        }
    }
    return q;
}

// Zero V and the frontier bitmaps, then set the seed of query q in V and in
// the bitmap that round 1 reads (rdone = rounds run so far in the launch).
template <typename E>
__device__ __forceinline__ void clean_prep(const PlainArgs<E> &a, uint64_t q, uint64_t rdone,
                                           uint64_t gtid, uint64_t gthreads) {
    uint64_t sw = ~0ull;
    uint32_t sb = 0;
    if (q < a.nq) {
        const uint32_t s = a.seeds[q];
        sw = s >> 5;
        sb = 1u << (s & 31);
    }
    const unsigned fin = (unsigned)(rdone % 3);
    for (uint64_t i = gtid; i < a.nw; i += gthreads) {
        const uint32_t val = i == sw ? sb : 0u;
        a.V[i] = val;
        a.F0[i] = fin == 0 ? val : 0u;
        a.F1[i] = fin == 1 ? val : 0u;
        a.F2[i] = fin == 2 ? val : 0u;
    }
}

template <typename E, int BLOCK>
__global__ void __launch_bounds__(BLOCK) plain_kernel(const PlainArgs<E> a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    E *s_pre = (E *)dyn_smem;
    E *s_rs = s_pre + ((1u << a.tile_log2) + 2u);
    __shared__ unsigned long long s_cnt, s_scan;
    __shared__ int s_flag;

    const bool b0 = blockIdx.x == 0 && threadIdx.x == 0;
    const uint64_t gtid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * BLOCK;
    unsigned epoch = 0;
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_scan = 0;
        epoch = ld_volatile_u32(&a.ctl->bar.gen);
    }
    uint64_t t_prev = b0 ? globaltimer_ns() : 0;
    __syncthreads();

    const uint64_t emask = (1ull << a.ebits) - 1ull;

    uint64_t rdone = 0;   // rounds run in this launch (selects the rotating buffers)
    uint64_t q = skip_trivial(a, 0, b0, t_prev);
    clean_prep(a, q, rdone, gtid, gthreads);
    if (!grid_barrier(&a.ctl->bar, &a.ctl->err, epoch, a.timeout_ns, &s_flag)) return;

    while (q < a.nq) {
        const uint32_t s = a.seeds[q];
        const uint32_t k = a.ks ? a.ks[q] : a.k_all;
        uint64_t mf = (uint64_t)(a.rp[s + 1] - a.rp[s]);   // out-edges of the frontier {s}
        uint64_t items = mf > 0 ? 1 : 0;
        uint64_t nf = 1;
        uint64_t count = 0, te = 0, bytes = 0, sum_mf = 0, visited = 1;
        uint32_t rounds = 0, pull_mask = 0;
        int prev = DIR_PUSH;
        for (uint32_t r = 1; r <= k && mf > 0; ++r) {
            ++rdone;
            const unsigned iin = (unsigned)((rdone - 1) % 3), iout = (unsigned)(rdone % 3);
            const unsigned izero = (unsigned)((rdone + 1) % 3);
            const unsigned qin = (unsigned)((rdone - 1) & 1), qout = (unsigned)(rdone & 1);
            int dir;
            if (r == 1) dir = a.direction == KHOP_DIR_PULL ? DIR_PULL : DIR_PUSH;
            else if (a.direction == KHOP_DIR_PUSH) dir = DIR_PUSH;
            else if (a.direction == KHOP_DIR_PULL) dir = DIR_PULL;
            else {
                const uint64_t mu = a.nnz - (sum_mf + mf);   // out-edges of unvisited vertices
                if (prev == DIR_PUSH)
                    dir = ((double)mf * (double)a.alpha > (double)mu) ? DIR_PULL : DIR_PUSH;
                else
                    dir = ((double)nf * (double)a.beta < (double)a.n && items <= a.pull_cap)
                              ? DIR_PUSH : DIR_PULL;
            }
            // Zero what round r+1 will write (read last in round r-1).
            uint32_t *Fz = sel3(a.F0, a.F1, a.F2, izero);
            for (uint64_t i = gtid; i < a.nw; i += gthreads) Fz[i] = 0u;
            if (b0) {
                unsigned long long *c = (unsigned long long *)a.ctl;
                c[izero] = 0ull;        // qpack
                c[3 + izero] = 0ull;    // nnew
                c[6 + izero] = 0ull;    // scanned
            }
            te += mf;
            Round<E> R;
            R.first = r == 1;
            R.last = r == k;
            R.seed = s;
            R.Fin = sel3(a.F0, a.F1, a.F2, iin);
            R.Fout = sel3(a.F0, a.F1, a.F2, iout);
            R.Qpre_in = qin ? a.Qpre1 : a.Qpre0;
            R.Qrs_in = qin ? a.Qrs1 : a.Qrs0;
            R.TF_in = qin ? a.TF1 : a.TF0;
            R.Qpre_out = qout ? a.Qpre1 : a.Qpre0;
            R.Qrs_out = qout ? a.Qrs1 : a.Qrs0;
            R.TF_out = qout ? a.TF1 : a.TF0;
            R.qpack_out = (unsigned long long *)a.ctl + iout;
            R.cap = dir == DIR_PUSH ? a.n : a.pull_cap;
            R.items_in = items;
            R.mf = mf;
            if (dir == DIR_PUSH) push_round<E, BLOCK>(a, R, s_pre, s_rs, &s_cnt);
            else pull_round<E, BLOCK>(a, R, &s_cnt, &s_scan);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_cnt) atomicAdd((unsigned long long *)a.ctl + 3 + iout, s_cnt);
                if (s_scan) atomicAdd((unsigned long long *)a.ctl + 6 + iout, s_scan);
                s_cnt = 0;
                s_scan = 0;
            }
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, epoch, a.timeout_ns, &s_flag)) return;
            const unsigned long long qp = ld_relaxed_u64((unsigned long long *)a.ctl + iout);
            const uint64_t nnew = ld_relaxed_u64((unsigned long long *)a.ctl + 3 + iout);
            const uint64_t scn = ld_relaxed_u64((unsigned long long *)a.ctl + 6 + iout);
            const uint64_t W = sizeof(E);
            const uint64_t items_out = R.last ? 0 : min((uint64_t)(qp >> a.ebits), R.cap);
            if (dir == DIR_PUSH)
                bytes += 4ull * mf + 2ull * W * ((r == 1 ? 1ull : items) + items_out);
            else
                bytes += 2ull * ((a.n + 7) / 8) + 2ull * W * (a.n - visited) + 4ull * scn +
                         2ull * W * items_out;
            sum_mf += mf;
            count += nnew;
            visited += nnew;
            nf = nnew;
            items = qp >> a.ebits;
            mf = R.last ? 0 : (qp & emask);
            prev = dir;
            rounds = r;
            if (dir == DIR_PULL && r <= 32) pull_mask |= 1u << (r - 1);
            if (b0 && a.per_hop && r < a.hop_stride) a.per_hop[q * a.hop_stride + r] = nnew;
            (void)nf;
        }
        if (b0) {
            const uint64_t now = globaltimer_ns();
            a.out[q] = count;
            if (a.out_te) a.out_te[q] = te;
            if (a.stats) {
                khop_query_stats st{t_prev, now, te, bytes, rounds, pull_mask};
                a.stats[q] = st;
            }
            if (a.per_hop) {
                if (a.hop_stride) a.per_hop[q * a.hop_stride] = 1ull;
                for (uint64_t r = (uint64_t)rounds + 1; r < a.hop_stride; ++r)
                    a.per_hop[q * a.hop_stride + r] = 0ull;
            }
            t_prev = now;
        }
        const uint64_t qn = skip_trivial(a, q + 1, b0, t_prev);
        clean_prep(a, qn, rdone, gtid, gthreads);
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, epoch, a.timeout_ns, &s_flag)) return;
        q = qn;
    }
}

template <typename E, int BLOCK>
int launch_block(khop_graph *g, PlainArgs<E> &a, size_t smem, cudaStream_t st) {
    const void *fn = (const void *)plain_kernel<E, BLOCK>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int grid = 0;
    int rc = cooperative_grid(fn, BLOCK, smem, g->tune.blocks_per_sm, g->num_sms, &grid);
    if (rc != KHOP_OK) return rc;
    e = cudaMemsetAsync(g->ctl, 0, offsetof(CtlBlock, err), st);
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BLOCK), args, smem, st);
    return cuda_status(e);
}

template <typename E>
int launch_typed(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint32_t k_all,
                 uint64_t nq, uint64_t *out, uint64_t *out_te, khop_query_stats *stats,
                 uint64_t *per_hop, uint32_t hop_stride, cudaStream_t st) {
    PlainArgs<E> a;
    a.n = g->n;
    a.nnz = g->nnz;
    a.nw = g->nw;
    a.symmetric = g->symmetric ? 1 : 0;
    a.rp = (const E *)g->rp;
    a.ci = g->ci;
    a.cp = (const E *)g->cp;
    a.ri = g->ri;
    a.V = g->V;
    a.F0 = g->F[0];
    a.F1 = g->F[1];
    a.F2 = g->F[2];
    a.Qpre0 = (E *)g->Qpre[0];
    a.Qpre1 = (E *)g->Qpre[1];
    a.Qrs0 = (E *)g->Qrs[0];
    a.Qrs1 = (E *)g->Qrs[1];
    a.TF0 = g->TF[0];
    a.TF1 = g->TF[1];
    a.ctl = g->ctl;
    a.seeds = seeds;
    a.ks = ks;
    a.k_all = k_all;
    a.nq = nq;
    a.out = out;
    a.out_te = out_te;
    a.stats = stats;
    a.per_hop = per_hop;
    a.hop_stride = per_hop ? hop_stride : 0u;
    a.direction = g->tune.direction;
    a.alpha = g->tune.alpha;
    a.beta = g->tune.beta;
    uint32_t tl = 0;
    while ((1u << tl) < (uint32_t)g->tune.push_tile) ++tl;
    a.tile_log2 = tl;
    a.ebits = g->ebits;
    a.pull_cap = g->tune.direction == KHOP_DIR_PULL
                     ? 0ull
                     : std::min<uint64_t>(g->n, (uint64_t)std::ceil((double)g->n / g->tune.beta) + 32);
    a.timeout_ns = g->timeout_ns;
    const size_t smem = 2 * ((size_t(1) << tl) + 2) * sizeof(E);
    switch (g->tune.block_threads) {
        case 256: return launch_block<E, 256>(g, a, smem, st);
        case 1024: return launch_block<E, 1024>(g, a, smem, st);
        default: return launch_block<E, 512>(g, a, smem, st);
    }
}

}  // namespace

int plain_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint32_t k_all,
                 uint64_t nq, uint64_t *out, uint64_t *out_te, khop_query_stats *stats,
                 uint64_t *per_hop, uint32_t hop_stride, cudaStream_t st) {
    if (g->ewidth == 4)
        return launch_typed<uint32_t>(g, seeds, ks, k_all, nq, out, out_te, stats, per_hop,
                                      hop_stride, st);
    return launch_typed<unsigned long long>(g, seeds, ks, k_all, nq, out, out_te, stats, per_hop,
                                            hop_stride, st);
}

}  // namespace khop
