// Bit-sliced batched k-hop count, 64 * LW lanes (LW = 1, 2 or 4 64-bit words).
//
// Up to 64 * LW queries share one traversal: every vertex v carries three lane
// words -- V[v] (lanes that have visited v), F_in[v] / F_out[v] (lanes
// whose frontier holds v this round / next round) -- so the (OR, AND)
// semiring of the single query becomes bitwise OR/AND on lane words:
//     F_out[w] = (OR over edges u -> w of F_in[u]) AND NOT V[w] AND active
// where `active` holds the lanes whose k has not been reached.  Lane j's count
// is the number of set j-bits of V at the end, minus its seed.
//
// Queries are grouped on the device into batches of 64 * LW by k (a counting
// sort by min(k, 63)), so the lanes of a batch mostly finish together.  One
// cooperative persistent launch then runs every batch: rounds of push
// (union-frontier queue, 64-bit atomicOr per lane word on V and F_out) or pull (lane-mask
// OR over the in-edges of every vertex some active lane has not visited, with
// an early exit once all those lanes are covered), chosen by a Beamer-style
// switch on the union frontier; then a harvest sweep counts the lane bits of
// V with bit-sliced counters and clears V for the next batch.
#include <algorithm>
#include <cmath>

#include "khop_internal.cuh"

namespace khop {
namespace {

enum { DIR_PUSH = 0, DIR_PULL = 1 };

constexpr int kBuckets = 64;         // batches are formed per bucket min(k, 63)
constexpr int kBlock = 512;          // threads per CTA of the batched kernels
constexpr int kPushUnroll = 4;
constexpr int kDeferEdges = 4096;    // longer in-lists go to the chunked pass
constexpr int kChunk = 4096;         // in-edges per chunk of the chunked pass
constexpr int kPlanes = 4;           // bit-sliced counter planes (up to 15 additions)
#ifdef KHOP_SCALAR_INDEX_LOADS
constexpr bool kVecIdx = false;      // the 4-byte-load build, kept for before/after measurements
#else
constexpr bool kVecIdx = true;       // pull: a lane reads its in-list four indices per 16-byte load
#endif
constexpr int kStage = 2048;
constexpr int kStagePosShift = 40;
constexpr unsigned long long kStageEdgeMask = (1ull << kStagePosShift) - 1ull;
constexpr uint32_t kEmpty = 0xffffffffu;

// A lane word: LW 64-bit words, lane l in bit l % 64 of word l / 64.
template <int LW>
struct __align__(8 * LW) Lanes {
    unsigned long long w[LW];
};

template <int LW>
__device__ __forceinline__ Lanes<LW> lzero() {
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = 0ull;
    return r;
}
template <int LW>
__device__ __forceinline__ bool lany(const Lanes<LW> &x) {
    unsigned long long o = 0ull;
#pragma unroll
    for (int j = 0; j < LW; ++j) o |= x.w[j];
    return o != 0ull;
}
template <int LW>
__device__ __forceinline__ Lanes<LW> land(const Lanes<LW> &a, const Lanes<LW> &b) {
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = a.w[j] & b.w[j];
    return r;
}
template <int LW>
__device__ __forceinline__ Lanes<LW> landnot(const Lanes<LW> &a, const Lanes<LW> &b) {   // a & ~b
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = a.w[j] & ~b.w[j];
    return r;
}
template <int LW>
__device__ __forceinline__ void lor_into(Lanes<LW> &a, const Lanes<LW> &b) {
#pragma unroll
    for (int j = 0; j < LW; ++j) a.w[j] |= b.w[j];
}
template <int LW>
__device__ __forceinline__ bool lcovers(const Lanes<LW> &acc, const Lanes<LW> &need) {   // need ⊆ acc
    bool r = true;
#pragma unroll
    for (int j = 0; j < LW; ++j) r = r && ((acc.w[j] & need.w[j]) == need.w[j]);
    return r;
}
template <int LW>
__device__ __forceinline__ Lanes<LW> lbit(int l) {
    Lanes<LW> r = lzero<LW>();
    r.w[l >> 6] = 1ull << (l & 63);
    return r;
}
// OR x into *p word by word (words of x that are zero are not touched);
// returns the old value of the touched words (zero for the others).
template <int LW>
__device__ __forceinline__ Lanes<LW> latomic_or(Lanes<LW> *p, const Lanes<LW> &x) {
    Lanes<LW> old;
#pragma unroll
    for (int j = 0; j < LW; ++j) old.w[j] = x.w[j] ? atomicOr(&p->w[j], x.w[j]) : 0ull;
    return old;
}
// The same OR without the old value (a fire-and-forget reduction).
template <int LW>
__device__ __forceinline__ void lred_or(Lanes<LW> *p, const Lanes<LW> &x) {
#pragma unroll
    for (int j = 0; j < LW; ++j)
        if (x.w[j])
            asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(&p->w[j]), "l"(x.w[j]) : "memory");
}
template <int LW>
__device__ __forceinline__ Lanes<LW> lload_relaxed(const Lanes<LW> *p) {
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = ld_relaxed_u64(&p->w[j]);
    return r;
}
template <int LW>
__device__ __forceinline__ Lanes<LW> lshfl(const Lanes<LW> &x, int src) {
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = __shfl_sync(FULL, x.w[j], src);
    return r;
}

template <typename E, int LW>
struct BatchArgs {
    uint64_t n, nnz;
    uint32_t nw;
    int symmetric;
    const E *rp;
    const uint32_t *ci;
    const E *cp;
    const uint32_t *ri;
    const uint32_t *noin;
    Lanes<LW> *V;
    Lanes<LW> *F0, *F1, *F2;
    uint32_t *Q0, *Q1;           // union-frontier queue: vertex ids
    E *Qpre0, *Qpre1;            // queue: out-edge prefix
    uint32_t *TF0, *TF1;         // first queue item of each push tile
    CtlBlock *ctl;
    unsigned long long *part;    // per-CTA lane counts [2][grid][64 * LW], by batch parity
    const uint32_t *seeds;
    const uint32_t *ks;
    uint64_t *out;
    const uint32_t *order;       // 64 * LW query indices per batch (kEmpty = unused lane)
    const unsigned long long *nbatches;
    uint32_t *hv;                // deferred pull vertices
    E *hend;
    Lanes<LW> *hneed, *hacc;
    uint64_t hcap;
    uint32_t *ch_item;           // chunks of the deferred in-lists
    E *ch_start;
    uint64_t ccap;
    uint64_t alpha_fx, beta_fx;   // Beamer's alpha and beta in 1/65536 units
    uint32_t tile_log2, ebits;
    int stage;
    uint64_t pull_cap;
    uint64_t timeout_ns;
    unsigned absent_at;      // testing: the last CTA skips its absent_at-th grid barrier (0 = never)
    uint32_t *S0, *S1;       // rolling batch: discovered vertices without out-edges, per round
                             // parity (null otherwise); with the queue they list every non-zero
                             // F_out entry
};

template <typename T>
__device__ __forceinline__ T sel3(T x0, T x1, T x2, unsigned i) {
    return i == 0 ? x0 : (i == 1 ? x1 : x2);
}

template <int LW>
struct Shared {
    unsigned long long cnt, mf, stage, limit, gbase, scan, unv;
    unsigned long long skipped;  // items not queued because the queue was past its cap
    int qfull;                   // this CTA saw the queue past its cap (pull rounds)
    unsigned long long slot[16];
    int flag;
    // lane table of the current batch
    uint32_t seed[64 * LW];
    uint32_t k[64 * LW];
    uint32_t qi[64 * LW];
    unsigned long long deg_pre[64 * LW + 1];   // round 1: exclusive prefix of the seeds' out-degrees
    uint32_t kmax;
};

template <typename E, int LW>
struct Round {
    bool first, last;
    bool precheck;               // read V before the atomic (once over 1/32 of n entered)
    Lanes<LW> act;               // lanes still running this round
    const Lanes<LW> *Fin;
    Lanes<LW> *Fout;
    const uint32_t *Q_in;
    const E *Qpre_in;
    const uint32_t *TF_in;
    uint32_t *Q_out;
    E *Qpre_out;
    uint32_t *TF_out;
    unsigned long long *qpack_out;
    uint64_t cap, items_in, mf;
    unsigned long long clean;    // one-word lanes: retired lanes whose V marks a pull sweep clears
    uint32_t *S_out;             // rolling batch: sink list of this round (or null)
};

template <typename E, int LW>
__device__ __forceinline__ void put_item(const BatchArgs<E, LW> &a, const Round<E, LW> &R, uint64_t pos,
                                         uint64_t pre, uint32_t w, E d) {
    if (pos >= R.cap) return;
    R.Q_out[pos] = w;
    R.Qpre_out[pos] = (E)pre;
    const uint64_t jf = (pre + (1ull << a.tile_log2) - 1ull) >> a.tile_log2;
    const uint64_t jl = (pre + (uint64_t)d - 1ull) >> a.tile_log2;
    for (uint64_t j = jf; j <= jl; ++j) R.TF_out[j] = (uint32_t)pos;
}

// Warp-collective: `isnew` marks a lane whose vertex w just entered the union
// frontier (with out-degree d > 0).  Union counts and out-edge sums go to the
// CTA; unless this is the last round w joins the next queue through the
// CTA's shared staging area (as in the single-query kernel).
template <typename E, int LW>
__device__ __forceinline__ void record(const BatchArgs<E, LW> &a, const Round<E, LW> &R, bool isnew,
                                       uint32_t w, E d, Shared<LW> &sh, uint32_t *st_w, E *st_pre,
                                       E *st_d) {
    const unsigned m = __ballot_sync(FULL, isnew);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    const E dd = isnew ? d : (E)0;
    const E incl = warp_inclusive_sum(dd);
    const E tot = __shfl_sync(FULL, incl, 31);
    if (lane == 0) {
        atomicAdd(&sh.cnt, (unsigned long long)__popc(m));
        atomicAdd(&sh.mf, (unsigned long long)tot);
    }
    if (R.last) return;
    const int leader = __ffs(m) - 1;
    const unsigned c = __popc(m);
    const uint64_t rank = (uint64_t)__popc(m & lanemask_lt());
    const uint64_t excl = (uint64_t)(incl - dd);
    unsigned long long old = 0;
    bool staged = false;
    if (a.stage) {
        if (lane == leader) {
            old = atomicAdd(&sh.stage, ((unsigned long long)c << kStagePosShift) + (unsigned long long)tot);
            if ((old >> kStagePosShift) + c > (unsigned long long)kStage) atomicMin(&sh.limit, old);
        }
        old = __shfl_sync(FULL, old, leader);
        staged = (old >> kStagePosShift) + c <= (unsigned long long)kStage;
    }
    const int qfull = __shfl_sync(FULL, *(volatile int *)&sh.qfull, 0);   // warp-uniform
    if (staged) {
        if (isnew) {
            const uint64_t p = (old >> kStagePosShift) + rank;
            st_w[p] = w;
            st_pre[p] = (E)((old & kStageEdgeMask) + excl);
            st_d[p] = d;
        }
    } else if (qfull) {
        // A pull round whose queue is already past its cap: the next round
        // pulls too, so only the item count is kept.
        if (lane == leader) atomicAdd(&sh.skipped, (unsigned long long)c);
    } else {
        if (lane == leader) {
            old = atomicAdd(R.qpack_out, ((unsigned long long)c << a.ebits) + (unsigned long long)tot);
            if ((old >> a.ebits) + c > R.cap) sh.qfull = 1;
        }
        old = __shfl_sync(FULL, old, leader);
        if (isnew)
            put_item(a, R, (old >> a.ebits) + rank, (old & ((1ull << a.ebits) - 1ull)) + excl, w, d);
    }
}

// Warp-collective: lanes with `is` append their vertex w to the round's sink
// list (rolling batches only; one global atomic per warp).
template <typename E, int LW>
__device__ __forceinline__ void sink_record(const BatchArgs<E, LW> &a, const Round<E, LW> &R, bool is,
                                            uint32_t w) {
    const unsigned m = __ballot_sync(FULL, is);
    if (m == 0u || R.S_out == nullptr) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&((RoundSlot *)R.qpack_out)->sinks, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    const uint64_t pos = base + (uint64_t)__popc(m & lanemask_lt());
    if (is && pos < a.n) R.S_out[pos] = w;
}

template <typename E, int LW>
__device__ __forceinline__ void flush_round(const BatchArgs<E, LW> &a, const Round<E, LW> &R, Shared<LW> &sh,
                                            uint32_t *st_w, E *st_pre, E *st_d,
                                            unsigned long long *slot_out) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long st = sh.stage;
        if (sh.limit < st) st = sh.limit;
        const uint32_t nst = (uint32_t)(st >> kStagePosShift);
        if (nst)
            sh.gbase = atomicAdd(R.qpack_out, ((unsigned long long)nst << a.ebits) +
                                                  (st & kStageEdgeMask));
        if (sh.skipped) atomicAdd(R.qpack_out, sh.skipped << a.ebits);
        sh.skipped = 0;
        sh.qfull = 0;
        if (sh.cnt) atomicAdd(slot_out + 1, sh.cnt);
        if (sh.scan) atomicAdd(slot_out + 2, sh.scan);
        if (sh.mf) atomicAdd(slot_out + 3, sh.mf);
        if (sh.unv) atomicAdd(slot_out + 4, sh.unv);
        sh.cnt = sh.mf = sh.scan = sh.unv = 0;
        sh.stage = 0;
        sh.limit = ~0ull;
        sh.flag = (int)nst;
    }
    __syncthreads();
    const uint32_t nst = (uint32_t)sh.flag;
    if (nst) {
        const uint64_t gpos = sh.gbase >> a.ebits;
        const uint64_t gpre = sh.gbase & ((1ull << a.ebits) - 1ull);
        for (uint32_t t = threadIdx.x; t < nst; t += kBlock)
            put_item(a, R, gpos + t, gpre + (uint64_t)st_pre[t], st_w[t], st_d[t]);
    }
}

// Visit w for the lanes in m: returns true if w entered the union frontier
// (its first frontier lane this round) and has out-edges; d = out-degree.
// The degree is read only for that first entry.  V is read before the
// atomic only once the union frontier has taken in over 1/32 of the vertices
// (before that nearly every target is new and the read only lengthens the
// chain).  In a batch's last round the lanes are ORed in without reading the
// old bits back (the harvest counts V), so no thread waits on the atomic.
template <typename E, int LW>
__device__ __forceinline__ bool visit(const BatchArgs<E, LW> &a, const Round<E, LW> &R, uint32_t w,
                                      const Lanes<LW> &m, E &d, Lanes<LW> &seen, bool &sink) {
    Lanes<LW> x = m;
    if (R.precheck) {
        x = landnot(m, a.V[w]);
        if (!lany(x)) return false;
    }
    if (R.last) {   // the harvest counts V: nothing needs the old bits
        lred_or(&a.V[w], x);
        return false;
    }
    const Lanes<LW> nb = landnot(x, latomic_or(&a.V[w], x));
    if (!lany(nb)) return false;
    lor_into(seen, nb);   // these lanes discovered a vertex this round
    // entry into the union frontier: a word of F_out[w] this call turned from
    // zero to non-zero.  With one word that is exactly one caller per vertex;
    // with LW words up to LW callers may queue w (extra work, same counts),
    // and at least one always does.
    const Lanes<LW> of = latomic_or(&R.Fout[w], nb);
    bool entered = false;
#pragma unroll
    for (int j = 0; j < LW; ++j) entered = entered || (nb.w[j] != 0ull && of.w[j] == 0ull);
    if (!entered) return false;
    d = a.rp[w + 1] - a.rp[w];
    sink = d == 0;
    return d > 0;
}

// Push round.  Round 1 expands the lanes' seeds straight from the lane table
// (item t = lane t, mask = its bit; a self-loop at the seed is skipped); later
// rounds expand the union-frontier queue with each item's lanes F_in[u] & act.
template <typename E, int LW>
__device__ __forceinline__ void push_round(const BatchArgs<E, LW> &a, const Round<E, LW> &R, E *s_pre,
                                           E *s_rs, Lanes<LW> *s_fm, uint32_t *s_u,
                                           Shared<LW> &sh, uint32_t *st_w, E *st_pre, E *st_d,
                                           Lanes<LW> &seen) {
    const uint32_t tl = a.tile_log2;
    const uint64_t T = 1ull << tl;
    const uint64_t ntiles = (R.mf + T - 1) >> tl;
    for (uint64_t j = blockIdx.x; j < ntiles; j += gridDim.x) {
        const uint64_t e0 = j << tl;
        const uint64_t e1 = min(e0 + T, R.mf);
        uint32_t nitems;
        if (R.first) {
            nitems = 64 * LW;
            if (threadIdx.x < 64 * LW) {
                const int l = threadIdx.x;
                const bool on = sh.qi[l] != kEmpty && ((R.act.w[l >> 6] >> (l & 63)) & 1ull);
                s_pre[l] = (E)sh.deg_pre[l];
                s_rs[l] = on ? a.rp[sh.seed[l]] : (E)0;
                s_fm[l] = on ? lbit<LW>(l) : lzero<LW>();
                s_u[l] = on ? sh.seed[l] : kEmpty;
            }
        } else {
            const uint64_t i0 = R.TF_in[j];
            const uint64_t il = (j + 1 < ntiles) ? (uint64_t)R.TF_in[j + 1] : R.items_in - 1;
            nitems = (uint32_t)(il - i0 + 1);
            for (uint32_t t = threadIdx.x; t < nitems; t += kBlock) {
                const uint32_t u = R.Q_in[i0 + t];
                s_pre[t] = R.Qpre_in[i0 + t];
                s_rs[t] = a.rp[u];
                s_fm[t] = land(R.Fin[u], R.act);
                s_u[t] = kEmpty;
            }
        }
        __syncthreads();
        uint32_t hint = 0;
        for (uint64_t base = e0; base < e1; base += (uint64_t)kBlock * kPushUnroll) {
            uint32_t w[kPushUnroll];
            Lanes<LW> m[kPushUnroll];
#pragma unroll
            for (int u = 0; u < kPushUnroll; ++u) {
                const uint64_t e = base + (uint64_t)u * kBlock + threadIdx.x;
                w[u] = 0;
                m[u] = lzero<LW>();
                if (e < e1) {
                    uint32_t lo = hint, hi = nitems - 1;   // largest item with prefix <= e
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if ((uint64_t)s_pre[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    hint = lo;
                    m[u] = s_fm[lo];
                    if (lany(m[u])) {
                        w[u] = a.ci[(uint64_t)s_rs[lo] + (e - (uint64_t)s_pre[lo])];
                        if (w[u] == s_u[lo]) m[u] = lzero<LW>();   // round 1: a seed's self-loop
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kPushUnroll; ++u) {
                E d = 0;
                bool sink = false;
                const bool isnew = lany(m[u]) && visit(a, R, w[u], m[u], d, seen, sink);
                record(a, R, isnew, w[u], d, sh, st_w, st_pre, st_d);
                if (R.S_out) sink_record(a, R, sink, w[u]);
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)x);
    const unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

template <int LW>
__device__ __forceinline__ Lanes<LW> warp_or(const Lanes<LW> &x) {
    Lanes<LW> r;
#pragma unroll
    for (int j = 0; j < LW; ++j) r.w[j] = warp_or64(x.w[j]);
    return r;
}

// Pull-round shape per lane-word width: in-edge loads in flight per lane
// (ilp) and the in-edges a lane scans alone before the warp helps
// (lane_edges).  Measured on the scale-21 R-MAT batches: two-word lanes gain
// most from eight loads in flight, one-word lanes from a longer solo scan.
template <int LW>
struct PullShape;
template <>
struct PullShape<1> {
    static constexpr int ilp = 4, lane_edges = 16;
};
template <>
struct PullShape<2> {
    static constexpr int ilp = 8, lane_edges = 8;
};
template <>
struct PullShape<4> {
    static constexpr int ilp = 8, lane_edges = 8;
};

// Pull round, sweep part.  Thread per vertex: need = act & ~V[v] (vertices
// without in-edges are skipped); the vertex ORs the frontier lanes F_in[u]
// of its in-neighbours until every needed lane is covered.  A lane first
// scans up to kLaneEdges in-edges itself (kPullILP loads in flight); the
// warp then takes the unresolved vertices one at a time, 32 * kPullILP
// in-edges per step, OR-reducing across the warp.  In-lists with more than
// kDeferEdges edges left are deferred to the chunked pass (pull_heavy).
template <typename E, int LW>
__device__ __forceinline__ void pull_round(const BatchArgs<E, LW> &a, const Round<E, LW> &R, Shared<LW> &sh,
                                           uint32_t *st_w, E *st_pre, E *st_d,
                                           unsigned long long *slot, Lanes<LW> &seen) {
    constexpr int kPullILP = PullShape<LW>::ilp, kLaneEdges = PullShape<LW>::lane_edges;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kBlock) >> 5;
    uint64_t scanned = 0, unv = 0;
    for (uint64_t i = gwarp; i < a.nw; i += nwarps) {
        const uint64_t v = (i << 5) + (uint64_t)lane;
        const uint32_t ni = a.noin[i];
        Lanes<LW> vv0 = lzero<LW>();
        if (v < a.n && !((ni >> lane) & 1u)) {
            vv0 = a.V[v];
            if (LW == 1 && (vv0.w[0] & R.clean)) {   // retired lanes' marks, cleared in passing
                vv0.w[0] &= ~R.clean;
                a.V[v] = vv0;
            }
        }
        Lanes<LW> need = lzero<LW>();
        if (v < a.n && !((ni >> lane) & 1u)) need = landnot(R.act, vv0);
        const bool needs = lany(need);
        const unsigned nmask = __ballot_sync(FULL, needs);
        if (nmask == 0u) continue;   // F_out was zeroed one round ahead
        unv += __popc(nmask);
        E b = 0, e = 0;
        if (needs) {
            b = a.cp[v];
            e = a.cp[v + 1];
        }
        Lanes<LW> acc = lzero<LW>();
        E pos = b;
        for (int it = 0; it < kLaneEdges / kPullILP; ++it) {
            const bool go = needs && pos < e && !lcovers(acc, need);
            if (!__any_sync(FULL, go)) break;
            uint32_t u[kPullILP];
            E took = 0;
            if (kVecIdx) {
                // the kPullILP/4 aligned 16-byte blocks of in-edge indices from
                // the block holding pos: one vector load per four indices (the
                // list's unaligned head and tail are masked off); the array's
                // last partial block is read index by index
                const E base = pos & ~(E)3;
                const E end = min(base + (E)kPullILP, e);
#pragma unroll
                for (int t = 0; t < kPullILP; t += 4) {
                    uint32_t q[4] = {kEmpty, kEmpty, kEmpty, kEmpty};
                    const E at = base + (E)t;
                    if (go && at < end) {
                        if ((uint64_t)at + 4 <= a.nnz) {
                            const uint4 v4 = *reinterpret_cast<const uint4 *>(a.ri + at);
                            q[0] = v4.x; q[1] = v4.y; q[2] = v4.z; q[3] = v4.w;
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if ((uint64_t)at + j < a.nnz) q[j] = a.ri[at + j];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const E x = at + (E)j;
                        u[t + j] = (go && x >= pos && x < end) ? q[j] : kEmpty;
                    }
                }
                if (go) took = end - pos;
            } else {
#pragma unroll
                for (int t = 0; t < kPullILP; ++t) u[t] = (go && pos + t < e) ? a.ri[pos + t] : kEmpty;
                if (go) took = min((E)kPullILP, e - pos);
            }
#pragma unroll
            for (int t = 0; t < kPullILP; ++t)
                if (u[t] != kEmpty) lor_into(acc, R.Fin[u[t]]);
            pos += took;
            scanned += (uint64_t)took;
        }
        const bool open = needs && pos < e && !lcovers(acc, need);
        const bool defer = open && (uint64_t)(e - pos) > (uint64_t)kDeferEdges;
        unsigned todo = __ballot_sync(FULL, open && !defer);
        while (todo) {
            const int L = __ffs(todo) - 1;
            const E vb = __shfl_sync(FULL, pos, L), ve = __shfl_sync(FULL, e, L);
            const Lanes<LW> nd = lshfl(need, L);
            const Lanes<LW> a0 = lshfl(acc, L);
            Lanes<LW> wacc = lzero<LW>();
            for (E c = vb; c < ve; c += (E)(32 * kPullILP)) {
                uint32_t u[kPullILP];
#pragma unroll
                for (int t = 0; t < kPullILP; ++t) {
                    const E idx = c + (E)(t * 32 + lane);
                    u[t] = idx < ve ? a.ri[idx] : kEmpty;
                }
#pragma unroll
                for (int t = 0; t < kPullILP; ++t)
                    if (u[t] != kEmpty) lor_into(wacc, R.Fin[u[t]]);
                if (lane == 0) scanned += (uint64_t)min((E)(32 * kPullILP), ve - c);
                Lanes<LW> f = warp_or(wacc);
                lor_into(f, a0);
                if (lcovers(f, nd)) break;
            }
            Lanes<LW> fin = warp_or(wacc);
            lor_into(fin, a0);
            if (lane == L) acc = fin;
            todo &= todo - 1u;
        }
        if (defer) {
            // the chunked pass finishes this vertex after the sweep
            const unsigned long long h = atomicAdd(slot + 5, 1ull);
            const uint64_t rest = (uint64_t)(e - pos);
            const uint64_t nch = (rest + kChunk - 1) / kChunk;
            const unsigned long long c0 = atomicAdd(slot + 6, (unsigned long long)nch);
            if (h < a.hcap && c0 + nch <= a.ccap) {
                a.hv[h] = (uint32_t)v;
                a.hend[h] = e;
                a.hneed[h] = need;
                a.hacc[h] = acc;
                for (uint64_t c = 0; c < nch; ++c) {
                    a.ch_item[c0 + c] = (uint32_t)h;
                    a.ch_start[c0 + c] = pos + (E)(c * kChunk);
                }
            } else {
                atomicOr(&a.ctl->err, (unsigned)KHOP_DEVERR_CAPACITY);
            }
        }
        const Lanes<LW> nb = defer ? lzero<LW>() : land(acc, need);
        const bool any_nb = lany(nb);
        lor_into(seen, nb);
        if (v < a.n && any_nb) {
            R.Fout[v] = nb;
            Lanes<LW> vv = vv0;
            lor_into(vv, nb);
            a.V[v] = vv;
        }
        E d = 0;
        if (any_nb && !R.last) d = a.symmetric ? e - b : a.rp[v + 1] - a.rp[v];
        record(a, R, any_nb && d > 0, (uint32_t)v, d, sh, st_w, st_pre, st_d);
        if (R.S_out) sink_record(a, R, any_nb && d == 0, (uint32_t)v);
    }
    scanned = warp_sum(scanned);
    if (lane == 0) {
        if (scanned) atomicAdd(&sh.scan, (unsigned long long)scanned);
        if (unv) atomicAdd(&sh.unv, (unsigned long long)unv);   // lane 0 counted whole words
    }
}

// Pull round, chunked pass over the deferred long in-lists: one warp per
// chunk of kChunk in-edges; each chunk's lane OR goes to its vertex's
// accumulator, and a chunk is skipped once its vertex has every needed lane.
template <typename E, int LW>
__device__ __forceinline__ void pull_chunks(const BatchArgs<E, LW> &a, const Round<E, LW> &R,
                                            uint64_t nchunks, Shared<LW> &sh) {
    constexpr int kPullILP = PullShape<LW>::ilp;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kBlock) >> 5;
    uint64_t scanned = 0;
    for (uint64_t c = gwarp; c < nchunks; c += nwarps) {
        const uint32_t h = a.ch_item[c];
        const Lanes<LW> nd = a.hneed[h];
        if (lcovers(lload_relaxed(&a.hacc[h]), nd)) continue;
        const E cb = a.ch_start[c];
        const E ce = min(cb + (E)kChunk, a.hend[h]);
        Lanes<LW> wacc = lzero<LW>();
        int steps = 0;
        for (E x = cb; x < ce; x += (E)(32 * kPullILP)) {
            uint32_t u[kPullILP];
#pragma unroll
            for (int t = 0; t < kPullILP; ++t) {
                const E idx = x + (E)(t * 32 + lane);
                u[t] = idx < ce ? a.ri[idx] : kEmpty;
            }
#pragma unroll
            for (int t = 0; t < kPullILP; ++t)
                if (u[t] != kEmpty) lor_into(wacc, R.Fin[u[t]]);
            if (lane == 0) scanned += (uint64_t)min((E)(32 * kPullILP), ce - x);
            if ((++steps & 7) == 0) {
                Lanes<LW> f = warp_or(wacc);
                lor_into(f, lload_relaxed(&a.hacc[h]));
                if (lcovers(f, nd)) break;
            }
        }
        const Lanes<LW> fin = land(warp_or(wacc), nd);
        if (lane == 0 && lany(fin)) latomic_or(&a.hacc[h], fin);
    }
    scanned = warp_sum(scanned);
    if (lane == 0 && scanned) atomicAdd(&sh.scan, (unsigned long long)scanned);
}

// Pull round, last part: settle the deferred vertices (thread per item).
template <typename E, int LW>
__device__ __forceinline__ void pull_settle(const BatchArgs<E, LW> &a, const Round<E, LW> &R,
                                            uint64_t nitems, Shared<LW> &sh, uint32_t *st_w,
                                            E *st_pre, E *st_d, Lanes<LW> &seen) {
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t iters = (nitems + gthreads - 1) / gthreads;   // uniform: record() is warp-wide
    for (uint64_t it = 0; it < iters; ++it) {
        const uint64_t h = gtid + it * gthreads;
        Lanes<LW> nb = lzero<LW>();
        uint32_t v = 0;
        E d = 0;
        if (h < nitems) {
            v = a.hv[h];
            nb = land(a.hacc[h], a.hneed[h]);
            a.hacc[h] = lzero<LW>();
            lor_into(seen, nb);
            R.Fout[v] = nb;
            if (lany(nb)) {
                Lanes<LW> vv = a.V[v];
                lor_into(vv, nb);
                a.V[v] = vv;
                if (!R.last) d = a.rp[v + 1] - a.rp[v];
            }
        }
        record(a, R, lany(nb) && d > 0, v, d, sh, st_w, st_pre, st_d);
        if (R.S_out) sink_record(a, R, lany(nb) && d == 0, v);
    }
}

// Harvest: per-lane popcount of V over all vertices, added into `row`
// (64 * LW lane totals); V is cleared on the way.  Each thread keeps, per
// lane word, kPlanes bit-sliced counters (plane i holds bit i of the 64 lane
// counts), adding one V word per step with a ripple carry; every 15 steps the
// warp sums its 32 threads' counters with a butterfly of bit-sliced adds
// (five shuffle levels, one more plane per level: at most 15 * 32 < 2^9),
// after which lane l reads the counts of bits l and l + 32 from the planes.
constexpr int kSumPlanes = kPlanes + 5;

template <int LW>
__device__ __forceinline__ void harvest(Lanes<LW> *V, uint64_t n, unsigned long long *row,
                                        unsigned *s_lane) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 64 * LW) s_lane[threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t iters = (n + gthreads - 1) / gthreads;   // uniform across the CTA
    unsigned long long p[kPlanes][LW];
#pragma unroll
    for (int i = 0; i < kPlanes; ++i)
#pragma unroll
        for (int j = 0; j < LW; ++j) p[i][j] = 0ull;
    for (uint64_t it = 0; it < iters; ++it) {
        const uint64_t v = gtid + it * gthreads;
        Lanes<LW> x = lzero<LW>();
        if (v < n) {
            x = V[v];
            if (lany(x)) V[v] = lzero<LW>();
        }
#pragma unroll
        for (int j = 0; j < LW; ++j) {
            unsigned long long y = x.w[j];
#pragma unroll
            for (int i = 0; i < kPlanes; ++i) {   // ripple-carry add of y into the planes
                const unsigned long long c = p[i][j] & y;
                p[i][j] ^= y;
                y = c;
            }
        }
        if ((it + 1) % ((1u << kPlanes) - 1u) == 0 || it + 1 == iters) {
#pragma unroll
            for (int j = 0; j < LW; ++j) {
                unsigned long long q[kSumPlanes];
#pragma unroll
                for (int i = 0; i < kSumPlanes; ++i) q[i] = i < kPlanes ? p[i][j] : 0ull;
#pragma unroll
                for (int lv = 0; lv < 5; ++lv) {   // q += q of lane ^ 2^lv
                    unsigned long long c = 0ull;
#pragma unroll
                    for (int i = 0; i < kSumPlanes; ++i) {
                        if (i > kPlanes + lv) break;   // planes above the current width are 0
                        const unsigned long long o = __shfl_xor_sync(FULL, q[i], 1 << lv);
                        const unsigned long long t = q[i] ^ o;
                        const unsigned long long cn = (q[i] & o) | (c & t);
                        q[i] = t ^ c;
                        c = cn;
                    }
                }
                unsigned lo = 0, hi = 0;
#pragma unroll
                for (int i = 0; i < kSumPlanes; ++i) {
                    lo |= (unsigned)((q[i] >> lane) & 1ull) << i;
                    hi |= (unsigned)((q[i] >> (lane + 32)) & 1ull) << i;
                }
#pragma unroll
                for (int i = 0; i < kPlanes; ++i) p[i][j] = 0ull;
                if (lo) atomicAdd(&s_lane[64 * j + lane], lo);
                if (hi) atomicAdd(&s_lane[64 * j + lane + 32], hi);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 64 * LW && s_lane[threadIdx.x])
        atomicAdd(row + threadIdx.x, (unsigned long long)s_lane[threadIdx.x]);
}

template <typename E, int LW>
__global__ void __launch_bounds__(kBlock, 2) batch_kernel(const BatchArgs<E, LW> a) {
    constexpr int B = 64 * LW;   // lanes per batch
    extern __shared__ __align__(32) unsigned char dyn_smem[];
    const uint32_t T2 = (1u << a.tile_log2) + 2u;
    Lanes<LW> *s_fm = (Lanes<LW> *)dyn_smem;                         // [T2]
    E *s_pre = (E *)(s_fm + T2);                                     // [T2]
    E *s_rs = s_pre + T2;                                            // [T2]
    uint32_t *s_u = (uint32_t *)(s_rs + T2);                         // [T2]
    uint32_t *st_w = s_u + T2;                                       // [kStage]
    E *st_pre = (E *)(st_w + kStage);                                // [kStage]
    E *st_d = st_pre + kStage;                                       // [kStage]
    __shared__ Shared<LW> sh;
    __shared__ unsigned s_lane[B];
    __shared__ unsigned long long s_deg[B];
    __shared__ uint32_t s_kx[B];
    __shared__ unsigned s_act[B / 32], s_more[B / 32];

    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    unsigned long long *slots = (unsigned long long *)a.ctl->slot;
    if (threadIdx.x == 0) {
        sh.cnt = sh.mf = sh.stage = sh.scan = sh.unv = 0;
        sh.limit = ~0ull;
        sh.skipped = 0;
        sh.qfull = 0;
    }
    // The frontier buffers rotate across launches: the buffer the next round
    // writes was zeroed by the previous round, and V was cleared by the last
    // harvest.  A launch that did not finish leaves `dirty` set, and the next
    // one starts from zeroed buffers.  Both words are read before the
    // prologue barrier and written only after it, so every CTA sees the same.
    BarState bsense = barrier_start(&a.ctl->bar, a.absent_at);
    const bool dirty = ld_volatile_u32(&a.ctl->dirty) != 0u;
    uint64_t rdone = dirty ? 0ull : *(volatile unsigned long long *)&a.ctl->rdone;
    if (gtid < 2ull * B) a.part[gtid] = 0ull;   // the two lane-total rows
    if (dirty)
        for (uint64_t v = gtid; v < a.n; v += gthreads) {
            a.F0[v] = lzero<LW>();
            a.F1[v] = lzero<LW>();
            a.F2[v] = lzero<LW>();
            a.V[v] = lzero<LW>();
        }
    if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns)) return;
    if (gtid == 0) a.ctl->dirty = 1u;
    const uint64_t nb_total = *a.nbatches;
    uint64_t bytes = 0, nrounds = 0, npull = 0;   // algorithmic HBM bytes, rounds run
    for (uint64_t b = 0; b < nb_total; ++b) {
        // lane table
        if (threadIdx.x < B) {
            const int l = threadIdx.x;
            const uint32_t qi = a.order[b * B + l];
            const uint32_t sd = qi != kEmpty ? a.seeds[qi] : 0u;
            const uint32_t kk = qi != kEmpty ? a.ks[qi] : 0u;
            sh.qi[l] = qi;
            sh.seed[l] = sd;
            sh.k[l] = kk;
            s_deg[l] = qi != kEmpty ? (unsigned long long)(a.rp[sd + 1] - a.rp[sd]) : 0ull;
            s_kx[l] = qi != kEmpty ? kk : 0u;
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive prefix of the seeds' out-degrees, max k
            constexpr int P = B / 32;
            const int t = threadIdx.x;
            unsigned long long d[P], sum = 0;
            uint32_t km = 0;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                d[j] = s_deg[t * P + j];
                sum += d[j];
                km = max(km, s_kx[t * P + j]);
            }
            const unsigned long long incl = warp_inclusive_sum(sum);
            unsigned long long acc = incl - sum;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                sh.deg_pre[t * P + j] = acc;
                acc += d[j];
            }
            if (t == 31) sh.deg_pre[B] = acc;
            km = __reduce_max_sync(FULL, km);
            if (t == 0) sh.kmax = km;
        }
        // seeds are visited by their own lanes
        if (blockIdx.x == 0 && threadIdx.x < B && sh.qi[threadIdx.x] != kEmpty)
            latomic_or(&a.V[sh.seed[threadIdx.x]], lbit<LW>(threadIdx.x));
        __syncthreads();
        const uint32_t kmax = sh.kmax;
        uint64_t mf = sh.deg_pre[B], items = B, nf = B;
        uint64_t entered = B;   // union-frontier entries so far (seeds included)
        int prev = DIR_PUSH;
        for (uint32_t r = 1; r <= kmax && mf > 0; ++r) {
            ++rdone;
            const unsigned iin = (unsigned)((rdone - 1) % 3), iout = (unsigned)(rdone % 3);
            const unsigned izero = (unsigned)((rdone + 1) % 3);
            const unsigned qin = (unsigned)((rdone - 1) & 1), qout = (unsigned)(rdone & 1);
            // lanes still running (k >= r) and whether any runs past r, by
            // ballots over the lane table (lane l = thread l), read by all
            if (threadIdx.x < B) {
                const int l = threadIdx.x;
                const bool on = sh.qi[l] != kEmpty && sh.k[l] >= r;
                const unsigned ma = __ballot_sync(FULL, on);
                const unsigned mm = __ballot_sync(FULL, on && sh.k[l] > r);
                if ((l & 31) == 0) {
                    s_act[l >> 5] = ma;
                    s_more[l >> 5] = mm;
                }
            }
            __syncthreads();
            Lanes<LW> act;
            bool last = true;
#pragma unroll
            for (int j = 0; j < LW; ++j) {
                act.w[j] = ((unsigned long long)s_act[2 * j + 1] << 32) | s_act[2 * j];
                last = last && s_more[2 * j] == 0u && s_more[2 * j + 1] == 0u;
            }
            __syncthreads();   // s_act / s_more are rewritten next round
            int dir = DIR_PUSH;
            if (r > 1) {
                if (prev == DIR_PUSH) dir = fx_gt(mf, a.alpha_fx, a.nnz) ? DIR_PULL : DIR_PUSH;
                else dir = (fx_lt(nf, a.beta_fx, a.n) && items <= a.pull_cap) ? DIR_PUSH : DIR_PULL;
            }
            Lanes<LW> *Fz = sel3(a.F0, a.F1, a.F2, izero);
            for (uint64_t v = gtid; v < a.n; v += gthreads) Fz[v] = lzero<LW>();
            if (gtid == 0) {
                slots[kSlotWords * izero + 0] = 0ull;
                slots[kSlotWords * izero + 1] = 0ull;
                slots[kSlotWords * izero + 2] = 0ull;
                slots[kSlotWords * izero + 3] = 0ull;
                slots[kSlotWords * izero + 4] = 0ull;
                slots[kSlotWords * izero + 5] = 0ull;
                slots[kSlotWords * izero + 6] = 0ull;
            }
            Round<E, LW> R;
            R.first = r == 1;
            R.last = last;
            R.precheck = entered * 32 > a.n;
            R.act = act;
            R.Fin = sel3(a.F0, a.F1, a.F2, iin);
            R.Fout = sel3(a.F0, a.F1, a.F2, iout);
            R.Q_in = qin ? a.Q1 : a.Q0;
            R.Qpre_in = qin ? a.Qpre1 : a.Qpre0;
            R.TF_in = qin ? a.TF1 : a.TF0;
            R.Q_out = qout ? a.Q1 : a.Q0;
            R.Qpre_out = qout ? a.Qpre1 : a.Qpre0;
            R.TF_out = qout ? a.TF1 : a.TF0;
            R.qpack_out = slots + kSlotWords * iout;
            R.cap = dir == DIR_PUSH ? a.n : a.pull_cap;
            R.items_in = items;
            R.mf = mf;
            R.clean = 0ull;
            R.S_out = nullptr;
            Lanes<LW> seen_unused = lzero<LW>();   // only the rolling kernel reads it
            if (dir == DIR_PUSH)
                push_round<E, LW>(a, R, s_pre, s_rs, s_fm, s_u, sh, st_w, st_pre, st_d, seen_unused);
            else {
                pull_round<E, LW>(a, R, sh, st_w, st_pre, st_d, slots + kSlotWords * iout, seen_unused);
                // deferred long in-lists (counts read after a barrier: uniform)
                if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, slots + kSlotWords * iout + 5,
                                  sh.slot + 5, 2, a.timeout_ns))
                    return;
                const uint64_t nitems = min((uint64_t)sh.slot[5], a.hcap);
                if (nitems) {
                    pull_chunks<E, LW>(a, R, min((uint64_t)sh.slot[6], a.ccap), sh);
                    if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0,
                                      a.timeout_ns))
                        return;
                    pull_settle<E, LW>(a, R, nitems, sh, st_w, st_pre, st_d, seen_unused);
                }
            }
            flush_round<E, LW>(a, R, sh, st_w, st_pre, st_d, slots + kSlotWords * iout);
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, slots + kSlotWords * iout, sh.slot, 5,
                              a.timeout_ns))
                return;
            // Algorithmic bytes (LB: bytes of a lane word): push: per frontier
            // vertex 2W row offsets + its lane word, per out-edge 4 + LB (edge
            // index, lane-word update); pull: LB n (visited sweep) + LB n (next
            // frontier) + 2W per vertex examined + (4 + LB) per in-edge scanned
            // (index, frontier gather).
            const uint64_t W = sizeof(E), LB = 8ull * LW;
            if (dir == DIR_PUSH)
                bytes += items * (2 * W + LB) + (4 + LB) * R.mf;
            else
                bytes += 2 * LB * a.n + 2 * W * sh.slot[4] + (4 + LB) * sh.slot[2];
            ++nrounds;
            if (dir == DIR_PULL) ++npull;
            nf = sh.slot[1];
            entered += nf;
            items = sh.slot[0] >> a.ebits;
            mf = last ? 0 : sh.slot[3];
            prev = dir;
        }
        // harvest the lane counts, clear V: every CTA adds its lane counts
        // into the row of this batch's parity; CTA 0 reads the totals after
        // the barrier and zeroes the row for batch b + 2.
        unsigned long long *row = a.part + (b & 1) * (uint64_t)B;
        harvest<LW>(a.V, a.n, row, s_lane);
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns)) return;
        if (blockIdx.x == 0 && threadIdx.x < B) {
            const int l = threadIdx.x;
            const unsigned long long tot = row[l];
            row[l] = 0ull;
            if (sh.qi[l] != kEmpty) a.out[sh.qi[l]] = tot - 1ull;   // minus the seed
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->pad[1] = bytes;
        a.ctl->pad[2] = nrounds;
        a.ctl->pad[3] = npull;
        a.ctl->rdone = rdone;
        __threadfence();
        a.ctl->dirty = 0u;
    }
}

// ===========================================================================
// Rolling 64-lane batch: continuous batching at round granularity.
//
// A request server keeps one traversal state per slot and runs it one round
// per launch ("step").  Lanes are independent bit positions, so lanes at
// different depths share a round: the round computes
//     F_out[w] = (OR over edges u -> w of F_in[u]) AND NOT V[w] AND act
// for every active lane at once, each advancing its own q_r by one hop.  A
// step (1) admits new requests into free lanes -- lane l with seed s gets
// V[s] |= l and F_in[s] |= l (its q_0 = {s}), and s joins the union-frontier
// queue unless it is in it already -- (2) runs one push or pull round for the
// active lanes, (3) counts each lane's discoveries of the round, retires the
// lanes whose k is reached or whose frontier came out empty (their counts are
// final) and zeroes the frontier buffer the round consumed.
//
// Every step's cost follows its frontier, not n: the queue and the sink list
// (discovered vertices without out-edges) together list every vertex whose
// F_out entry the round set, so the discoveries are counted and the spent F_in
// zeroed by walking them.  Only a pull round whose queue overflowed (more
// discoveries than a switch back to push would take) leaves its buffer
// "dense", handled by full sweeps.  F entries are never cleared bit by bit
// (an entry is non-zero exactly when its vertex is listed), so a retired
// lane's bits stay in the next frontier, masked off by `act`, until that
// buffer is zeroed one round later; the host reuses the lane after that.  Its
// visited marks are cleared lazily: the next pull round (which reads V of
// every vertex with in-edges) clears them in passing, its seed's mark is
// cleared at once, and a step asked for a dense clean sweeps V.  The state
// between steps -- queue size, out-edges, union frontier, direction, which
// buffers are dense, the lanes' seeds and running counts -- stays on the
// device.

// Control-block words the rolling state keeps between steps.
enum { RS_MF = 0, RS_ITEMS, RS_NF, RS_ENTERED, RS_PREV, RS_DEAD, RS_DENSE, RS_NSINK, RS_WORDS };

// The vertices whose F entry a round set: its queue Q[0..nq) then its sink
// list S[0..ns) -- or, when `dense` (the queue overflowed), all n vertices.
struct Listed {
    const uint32_t *Q, *S;
    uint64_t nq, ns;
    bool dense;
    __device__ __forceinline__ uint64_t total(uint64_t n) const { return dense ? n : nq + ns; }
    __device__ __forceinline__ uint64_t at(uint64_t x) const {
        return dense ? x : (x < nq ? (uint64_t)Q[x] : (uint64_t)S[x - nq]);
    }
};

// Per-lane bit counts of F over the listed vertices, added into row[64]
// (bit-sliced planes as in harvest()); with `zero`, the entries are zeroed
// after they are read.
__device__ __forceinline__ void roll_count(Lanes<1> *F, const Listed &L, uint64_t n, bool zero,
                                           unsigned long long *row, unsigned *s_lane) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 64) s_lane[threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t total = L.total(n);
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t iters = (total + gthreads - 1) / gthreads;   // uniform across the grid
    unsigned long long p[kPlanes];
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) p[i] = 0ull;
    for (uint64_t it = 0; it < iters; ++it) {
        const uint64_t x = gtid + it * gthreads;
        unsigned long long y = 0ull;
        if (x < total) {
            const uint64_t w = L.at(x);
            y = F[w].w[0];
            if (zero && y) F[w].w[0] = 0ull;
        }
#pragma unroll
        for (int i = 0; i < kPlanes; ++i) {   // ripple-carry add of y into the planes
            const unsigned long long c = p[i] & y;
            p[i] ^= y;
            y = c;
        }
        if ((it + 1) % ((1u << kPlanes) - 1u) == 0 || it + 1 == iters) {
            unsigned long long q[kSumPlanes];
#pragma unroll
            for (int i = 0; i < kSumPlanes; ++i) q[i] = i < kPlanes ? p[i] : 0ull;
#pragma unroll
            for (int lv = 0; lv < 5; ++lv) {   // q += q of lane ^ 2^lv
                unsigned long long c = 0ull;
#pragma unroll
                for (int i = 0; i < kSumPlanes; ++i) {
                    if (i > kPlanes + lv) break;
                    const unsigned long long o = __shfl_xor_sync(FULL, q[i], 1 << lv);
                    const unsigned long long t = q[i] ^ o;
                    const unsigned long long cn = (q[i] & o) | (c & t);
                    q[i] = t ^ c;
                    c = cn;
                }
            }
            unsigned lo = 0, hi = 0;
#pragma unroll
            for (int i = 0; i < kSumPlanes; ++i) {
                lo |= (unsigned)((q[i] >> lane) & 1ull) << i;
                hi |= (unsigned)((q[i] >> (lane + 32)) & 1ull) << i;
            }
#pragma unroll
            for (int i = 0; i < kPlanes; ++i) p[i] = 0ull;
            if (lo) atomicAdd(&s_lane[lane], lo);
            if (hi) atomicAdd(&s_lane[lane + 32], hi);
        }
    }
    __syncthreads();
    if (threadIdx.x < 64 && s_lane[threadIdx.x])
        atomicAdd(row + threadIdx.x, (unsigned long long)s_lane[threadIdx.x]);
}

// Zero F at the listed vertices.
__device__ __forceinline__ void roll_zero(Lanes<1> *F, const Listed &L, uint64_t n) {
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t total = L.total(n);
    for (uint64_t x = gtid; x < total; x += gthreads) F[L.at(x)].w[0] = 0ull;
}

template <typename E>
__global__ void __launch_bounds__(kBlock, 2) roll_kernel(const BatchArgs<E, 1> a, const RollPlan plan,
                                                        RollResult *res) {
    constexpr int LW = 1;
    extern __shared__ __align__(32) unsigned char dyn_smem[];
    const uint32_t T2 = (1u << a.tile_log2) + 2u;
    Lanes<LW> *s_fm = (Lanes<LW> *)dyn_smem;                         // [T2]
    E *s_pre = (E *)(s_fm + T2);                                     // [T2]
    E *s_rs = s_pre + T2;                                            // [T2]
    uint32_t *s_u = (uint32_t *)(s_rs + T2);                         // [T2]
    uint32_t *st_w = s_u + T2;                                       // [kStage]
    E *st_pre = (E *)(st_w + kStage);                                // [kStage]
    E *st_d = st_pre + kStage;                                       // [kStage]
    __shared__ Shared<LW> sh;
    __shared__ unsigned s_lane[64];
    __shared__ unsigned long long s_seen;
    __shared__ unsigned long long s_st[RS_WORDS];

    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    unsigned long long *slots = (unsigned long long *)a.ctl->slot;
    unsigned long long *hs = a.ctl->handoff;   // RS_* words
    unsigned long long *total = a.part;        // [64] running count of each lane
    unsigned long long *lseed = a.part + 64;   // [64] seed of each lane in use
    const uint64_t t_start = (blockIdx.x == 0 && threadIdx.x == 0) ? globaltimer_ns() : 0ull;
    if (threadIdx.x == 0) {
        sh.cnt = sh.mf = sh.stage = sh.scan = sh.unv = 0;
        sh.limit = ~0ull;
        sh.skipped = 0;
        sh.qfull = 0;
        s_seen = 0ull;
    }
    BarState bsense = barrier_start(&a.ctl->bar, a.absent_at);
    // A step that did not finish leaves `dirty` set; the host asks for a reset
    // after it gave a step up.  Either way the state starts from zero.
    const bool fresh = plan.reset != 0u || ld_volatile_u32(&a.ctl->dirty) != 0u;
    uint64_t rdone = fresh ? 0ull : *(volatile unsigned long long *)&a.ctl->rdone;
    if (fresh) {
        for (uint64_t v = gtid; v < a.n; v += gthreads) {
            a.V[v] = lzero<LW>();
            a.F0[v] = lzero<LW>();
            a.F1[v] = lzero<LW>();
            a.F2[v] = lzero<LW>();
        }
        if (gtid < 128) a.part[gtid] = 0ull;
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns))
            return;
    } else if (plan.clean_dense && plan.clean) {
        // the retired lanes' visited marks, everywhere (admission below only
        // sets bits of other lanes, so both may run at once)
        for (uint64_t v = gtid; v < a.n; v += gthreads)
            if (a.V[v].w[0] & plan.clean) atomicAnd(&a.V[v].w[0], ~plan.clean);
    }
    // (1) admission, by the first warp of CTA 0: new lanes into V, F_in and
    // the union-frontier queue the round reads.
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long st[RS_WORDS];
#pragma unroll
        for (int i = 0; i < RS_WORDS; ++i) st[i] = fresh ? 0ull : hs[i];
        Lanes<LW> *Fin = sel3(a.F0, a.F1, a.F2, (unsigned)(rdone % 3));
        Round<E, LW> R;
        R.Q_out = (rdone & 1) ? a.Q1 : a.Q0;
        R.Qpre_out = (rdone & 1) ? a.Qpre1 : a.Qpre0;
        R.TF_out = (rdone & 1) ? a.TF1 : a.TF0;
        R.cap = a.n;
        unsigned long long dead = 0ull;
        for (uint32_t base = 0; base < plan.nadmit; base += 32) {
            const uint32_t t = base + (uint32_t)lane;
            const bool on = t < plan.nadmit && t < 64u;
            const uint32_t l = on ? plan.lane[t] & 63u : 0u, s = on ? plan.seed[t] : 0u;
            E d = 0;
            bool ni = false;
            if (on) {
                d = a.rp[s + 1] - a.rp[s];
                const unsigned long long bit = 1ull << l;
                total[l] = 0ull;
                lseed[l] = s;
                if (d == 0) {
                    dead |= bit;
                } else {
                    atomicOr(&a.V[s].w[0], bit);
                    ni = atomicOr(&Fin[s].w[0], bit) == 0ull;   // s enters the union frontier
                }
            }
            const E dd = ni ? d : (E)0;
            const E incl = warp_inclusive_sum(dd);
            const unsigned m = __ballot_sync(FULL, ni);
            if (ni)
                put_item(a, R, st[RS_ITEMS] + (uint64_t)__popc(m & lanemask_lt()),
                         st[RS_MF] + (uint64_t)(incl - dd), s, d);
            st[RS_ITEMS] += (unsigned long long)__popc(m);
            st[RS_MF] += (unsigned long long)__shfl_sync(FULL, incl, 31);
            st[RS_NF] += (unsigned long long)__popc(m);
            st[RS_ENTERED] += (unsigned long long)__popc(m);
        }
        dead = warp_or64(dead);
        if (lane == 0) {
            st[RS_DEAD] = dead;
#pragma unroll
            for (int i = 0; i < RS_WORDS; ++i) hs[i] = st[i];
        }
    }
    if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, hs, s_st, RS_WORDS, a.timeout_ns)) return;
    if (gtid == 0) a.ctl->dirty = 1u;
    uint64_t mf = s_st[RS_MF], items = s_st[RS_ITEMS], nf = s_st[RS_NF], entered = s_st[RS_ENTERED];
    int prev = (int)s_st[RS_PREV];
    const unsigned long long dead = s_st[RS_DEAD];
    unsigned dense = (unsigned)s_st[RS_DENSE];       // bit b: F buffer b is not listed by its queue
    const unsigned long long act = plan.act & ~dead;
    // (2) one round for the active lanes
    const bool run = act != 0ull && mf > 0;
    const uint64_t items_in = items, nsink_in = s_st[RS_NSINK];
    uint64_t nsink_out = 0;
    unsigned long long seen_all = 0ull, bytes = 0ull, pulled = 0ull;
    bool cleaned = plan.clean_dense != 0u;
    if (run) {
        ++rdone;
        const unsigned iin = (unsigned)((rdone - 1) % 3), iout = (unsigned)(rdone % 3);
        const unsigned qin = (unsigned)((rdone - 1) & 1), qout = (unsigned)(rdone & 1);
        // Direction.  A pull exits a vertex's in-list early only once every
        // lane that still needs the vertex is covered, and lanes that joined
        // recently (small frontiers) almost never are: with lanes at widely
        // mixed depths a pull scans nearly every in-edge.  So a rolling batch
        // pushes unless the plan allows Beamer's switch (the host allows it
        // when its lanes' depths are close); a queue that overflowed in a
        // pull forces the next round to pull too.
        int dir = DIR_PUSH;
        if (prev == DIR_PULL && items > a.pull_cap) dir = DIR_PULL;
        else if (plan.pull_ok) {
            if (prev == DIR_PUSH) dir = fx_gt(mf, a.alpha_fx, a.nnz) ? DIR_PULL : DIR_PUSH;
            else dir = (fx_lt(nf, a.beta_fx, a.n) && items <= a.pull_cap) ? DIR_PUSH : DIR_PULL;
        }
        // (the round's counter slot was zeroed with the control block at launch)
        Round<E, LW> R;
        R.first = false;
        R.last = false;
        R.precheck = entered * 32 > a.n;
        R.act.w[0] = act;
        R.Fin = sel3(a.F0, a.F1, a.F2, iin);
        R.Fout = sel3(a.F0, a.F1, a.F2, iout);
        R.Q_in = qin ? a.Q1 : a.Q0;
        R.Qpre_in = qin ? a.Qpre1 : a.Qpre0;
        R.TF_in = qin ? a.TF1 : a.TF0;
        R.Q_out = qout ? a.Q1 : a.Q0;
        R.Qpre_out = qout ? a.Qpre1 : a.Qpre0;
        R.TF_out = qout ? a.TF1 : a.TF0;
        R.qpack_out = slots + kSlotWords * iout;
        R.cap = dir == DIR_PUSH ? a.n : a.pull_cap;
        R.items_in = items;
        R.mf = mf;
        R.clean = dir == DIR_PULL ? plan.clean : 0ull;
        R.S_out = qout ? a.S1 : a.S0;
        Lanes<LW> seen = lzero<LW>();
        if (dir == DIR_PUSH) {
            push_round<E, LW>(a, R, s_pre, s_rs, s_fm, s_u, sh, st_w, st_pre, st_d, seen);
        } else {
            pull_round<E, LW>(a, R, sh, st_w, st_pre, st_d, slots + kSlotWords * iout, seen);
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, slots + kSlotWords * iout + 5,
                              sh.slot + 5, 2, a.timeout_ns))
                return;
            const uint64_t nitems = min((uint64_t)sh.slot[5], a.hcap);
            if (nitems) {
                pull_chunks<E, LW>(a, R, min((uint64_t)sh.slot[6], a.ccap), sh);
                if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0,
                                  a.timeout_ns))
                    return;
                pull_settle<E, LW>(a, R, nitems, sh, st_w, st_pre, st_d, seen);
            }
        }
        const unsigned long long sw = warp_or64(seen.w[0]);
        if ((threadIdx.x & 31) == 0 && sw) atomicOr(&s_seen, sw);
        flush_round<E, LW>(a, R, sh, st_w, st_pre, st_d, slots + kSlotWords * iout);
        if (threadIdx.x == 0 && s_seen) atomicOr(slots + kSlotWords * iout + 7, s_seen);
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, slots + kSlotWords * iout, sh.slot, 9,
                          a.timeout_ns))
            return;
        const uint64_t W = sizeof(E), LB = 8ull;
        if (dir == DIR_PUSH) {
            bytes = items * (2 * W + LB) + (4 + LB) * mf;
        } else {
            bytes = 2 * LB * a.n + 2 * W * sh.slot[4] + (4 + LB) * sh.slot[2];
            pulled = 1ull;
            cleaned = true;   // the sweep read V of every vertex with in-edges
        }
        seen_all = sh.slot[7];
        nsink_out = sh.slot[8];
        nf = sh.slot[1];
        entered += nf;
        const uint64_t counted = sh.slot[0] >> a.ebits;   // queue entries of the round (stored or not)
        items = counted;
        mf = sh.slot[3];
        prev = dir;
        // the output buffer is listed by its queue unless the queue overflowed
        if (counted > R.cap) dense |= 1u << iout;
        else dense &= ~(1u << iout);
    }
    // (3) retire: k reached, or nothing discovered this round (the lane's
    // frontier is empty, so its count is final), or a seed without out-edges
    const unsigned long long retire = (plan.fin & act) | (act & ~seen_all) | dead;
    const bool idle = (act & ~retire) == 0ull;   // no lane continues: the next step starts clean
    if (run) {
        const unsigned iin = (unsigned)((rdone - 1) % 3), iout = (unsigned)(rdone % 3);
        const unsigned pin = (unsigned)((rdone - 1) & 1), pout = (unsigned)(rdone & 1);
        const Listed Lout{pout ? a.Q1 : a.Q0, pout ? a.S1 : a.S0, items, nsink_out, ((dense >> iout) & 1u) != 0u};
        const Listed Lin{pin ? a.Q1 : a.Q0, pin ? a.S1 : a.S0, items_in, nsink_in, ((dense >> iin) & 1u) != 0u};
        // the round's discoveries per lane (and, with no lane left, the buffer
        // is zeroed on the way); the consumed frontier is zeroed (it is
        // written again two rounds on)
        roll_count(sel3(a.F0, a.F1, a.F2, iout), Lout, a.n, idle, total, s_lane);
        roll_zero(sel3(a.F0, a.F1, a.F2, iin), Lin, a.n);
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns))
            return;
    } else if (idle && (items_in || nsink_in)) {
        // no round ran and no lane continues: zero the frontier the next round would read
        const unsigned icur = (unsigned)(rdone % 3), pcur = (unsigned)(rdone & 1);
        const Listed Lcur{pcur ? a.Q1 : a.Q0, pcur ? a.S1 : a.S0, items_in, nsink_in, ((dense >> icur) & 1u) != 0u};
        roll_zero(sel3(a.F0, a.F1, a.F2, icur), Lcur, a.n);
        if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns))
            return;
    }
    if (run) dense &= ~(1u << (unsigned)((rdone - 1) % 3));
    if (blockIdx.x != 0) return;
    if (threadIdx.x < 64) {
        const int l = threadIdx.x;
        if ((retire >> l) & 1ull) {
            res->count[l] = total[l];
            total[l] = 0ull;
            if (!((dead >> l) & 1ull)) {   // its seed's mark goes now, the rest lazily
                const uint64_t sd = lseed[l];
                atomicAnd(&a.V[sd].w[0], ~(1ull << l));
            }
        }
    }
    __syncthreads();   // the counts are written before `done`
    if (threadIdx.x == 0) {
        hs[RS_MF] = idle ? 0ull : mf;
        hs[RS_ITEMS] = idle ? 0ull : items;
        hs[RS_NF] = idle ? 0ull : nf;
        hs[RS_ENTERED] = idle ? 0ull : entered;
        hs[RS_PREV] = idle ? (unsigned long long)DIR_PUSH : (unsigned long long)prev;
        hs[RS_DEAD] = 0ull;
        hs[RS_DENSE] = idle ? 0ull : dense;   // no lane left: every buffer is zero
        hs[RS_NSINK] = idle ? 0ull : (run ? nsink_out : nsink_in);
        a.ctl->rdone = rdone;
        res->retired = retire;
        res->cleaned = cleaned ? plan.clean : 0ull;
        res->rdone = rdone;
        res->idle = idle ? 1ull : 0ull;
        res->union_nf = nf;
        res->bytes = bytes;
        res->pulled = pulled;
        res->t_start_ns = t_start;
        res->t_end_ns = globaltimer_ns();
        __threadfence_system();
        a.ctl->dirty = 0u;
        res->done = 1ull;
    }
}

// Group the queries into batches of 64 * LW by min(k, 63); answer k = 0 and
// seeds >= n directly.  One CTA: histogram, padded exclusive scan, scatter.
template <int LW>
__global__ void __launch_bounds__(1024) group_kernel(const uint32_t *seeds, const uint32_t *ks,
                                                     uint64_t nq, uint64_t n, uint64_t *out,
                                                     uint32_t *order, uint64_t order_cap,
                                                     unsigned long long *nbatches, unsigned *err) {
    __shared__ unsigned long long cnt[kBuckets], base[kBuckets], cur[kBuckets];
    if (threadIdx.x < kBuckets) cnt[threadIdx.x] = cur[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < nq; i += blockDim.x) {
        const uint32_t s = seeds[i], k = ks[i];
        if (s >= n) {
            out[i] = ~0ull;
            atomicOr(err, (unsigned)KHOP_DEVERR_SEED);
        } else if (k == 0) {
            out[i] = 0ull;
        } else {
            atomicAdd(&cnt[min(k, (uint32_t)kBuckets - 1)], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int b = 0; b < kBuckets; ++b) {
            base[b] = acc;
            acc += (cnt[b] + 64 * LW - 1) / (64 * LW) * (64 * LW);
        }
        *nbatches = acc / (64 * LW);
    }
    __syncthreads();
    const unsigned long long total = *nbatches * (64 * LW);
    for (uint64_t i = threadIdx.x; i < total && i < order_cap; i += blockDim.x) order[i] = kEmpty;
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < nq; i += blockDim.x) {
        const uint32_t s = seeds[i], k = ks[i];
        if (s >= n || k == 0) continue;
        const int bk = (int)min(k, (uint32_t)kBuckets - 1);
        const unsigned long long p = base[bk] + atomicAdd(&cur[bk], 1ull);
        if (p < order_cap) order[p] = (uint32_t)i;
    }
}

// Kernel arguments over a batch state.
template <typename E, int LW>
BatchArgs<E, LW> make_args(khop_graph *g, BatchState &bs, const uint32_t *seeds, const uint32_t *ks,
                           uint64_t *out, const uint32_t *order, const unsigned long long *nbatches,
                           bool take_test_switch = true) {
    BatchArgs<E, LW> a;
    a.n = g->n;
    a.nnz = g->nnz;
    a.nw = g->nw;
    a.symmetric = g->symmetric ? 1 : 0;
    a.rp = (const E *)g->rp;
    a.ci = g->ci;
    a.cp = (const E *)g->cp;
    a.ri = g->ri;
    a.noin = g->noin;
    a.V = (Lanes<LW> *)bs.V;
    a.F0 = (Lanes<LW> *)bs.F[0];
    a.F1 = (Lanes<LW> *)bs.F[1];
    a.F2 = (Lanes<LW> *)bs.F[2];
    a.Q0 = bs.Q[0];
    a.Q1 = bs.Q[1];
    a.Qpre0 = (E *)bs.Qpre[0];
    a.Qpre1 = (E *)bs.Qpre[1];
    a.TF0 = bs.TF[0];
    a.TF1 = bs.TF[1];
    a.ctl = bs.ctl;
    a.part = bs.part;
    a.seeds = seeds;
    a.ks = ks;
    a.out = out;
    a.order = order;
    a.nbatches = nbatches;
    a.hv = bs.hv;
    a.hend = (E *)bs.hend;
    a.hneed = (Lanes<LW> *)bs.hneed;
    a.hacc = (Lanes<LW> *)bs.hacc;
    a.hcap = bs.hcap;
    a.ch_item = bs.ch_item;
    a.ch_start = (E *)bs.ch_start;
    a.ccap = bs.ccap;
    a.alpha_fx = factor_fx16(g->tune.batch_alpha);
    a.beta_fx = factor_fx16(g->tune.batch_beta);
    uint32_t tl = 0;
    while ((1u << tl) < (uint32_t)g->tune.batch_push_tile) ++tl;
    if (LW == 2 && tl > 12) tl = 12;   // 128 lanes: tiles of at most 4096 edges fit shared memory
    if (LW == 4 && tl > 11) tl = 11;   // 256 lanes: at most 2048
    a.tile_log2 = tl;
    a.ebits = g->ebits;
    a.stage = g->nnz < (1ull << kStagePosShift) ? 1 : 0;
    a.pull_cap = std::min<uint64_t>(g->n, (uint64_t)std::ceil((double)g->n / g->tune.batch_beta) + 32);
    a.timeout_ns = g->timeout_ns;
    a.S0 = bs.S[0];
    a.S1 = bs.S[1];
    a.absent_at = 0;
    if (take_test_switch) {
        a.absent_at = g->absent_at;   // one launch only
        g->absent_at = 0;
    }
    return a;
}

// Cooperative launch of the batch kernel over `bs`; grid_ctas = 0 fills the
// GPU, otherwise at most that many CTAs (so that several run side by side).
template <typename E, int LW>
int launch_kernel(khop_graph *g, BatchState &bs, BatchArgs<E, LW> &a, int grid_ctas, cudaStream_t st) {
    const size_t T2 = (size_t(1) << a.tile_log2) + 2;
    const size_t smem = T2 * (8 * LW + 2 * sizeof(E) + 4) + kStage * (4 + 2 * sizeof(E));
    const void *fn = (const void *)batch_kernel<E, LW>;
    int grid = 0;
    int rc = launch_shape(fn, kBlock, smem, 0, g->num_sms, &grid);
    if (rc != KHOP_OK) return rc;
    cudaError_t e;
    if (grid_ctas > 0 && grid_ctas < grid) grid = grid_ctas;
    if ((uint64_t)grid > bs.part_rows) return KHOP_EINVAL;
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, smem, st);
    return cuda_status(e);
}

template <typename E, int LW>
int launch_typed(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st) {
    BatchState &bs = LW == 4 ? g->batch4 : (LW == 2 ? g->batch2 : g->batch);
    // order: nq plus up to 64 * LW - 1 padding lanes per bucket
    const uint64_t need = nq + 64ull * LW * kBuckets;
    if (bs.order_cap < need) {
        cudaFree(bs.order);
        bs.order = nullptr;
        bs.order_cap = 0;
        cudaError_t e = cudaMalloc(&bs.order, need * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_status(e);
        bs.order_cap = need;
    }
    cudaError_t e = cudaMemsetAsync(bs.ctl, 0, offsetof(CtlBlock, err), st);
    if (e != cudaSuccess) return cuda_status(e);
    group_kernel<LW><<<1, 1024, 0, st>>>(seeds, ks, nq, g->n, out, bs.order, bs.order_cap,
                                         (unsigned long long *)&bs.ctl->pad[0], &bs.ctl->err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    BatchArgs<E, LW> a = make_args<E, LW>(g, bs, seeds, ks, out, bs.order,
                                          (const unsigned long long *)&bs.ctl->pad[0]);
    return launch_kernel<E, LW>(g, bs, a, 0, st);
}


template <typename E>
int roll_typed(khop_graph *g, BatchState &bs, const RollPlan &plan, RollResult *res, int grid_ctas,
               cudaStream_t st) {
    if (bs.lw != 1) return KHOP_EINVAL;
    BatchArgs<E, 1> a = make_args<E, 1>(g, bs, nullptr, nullptr, nullptr, nullptr, nullptr, false);
    if (!a.S0 || !a.S1) return KHOP_EINVAL;   // a rolling state has sink lists
    const size_t T2 = (size_t(1) << a.tile_log2) + 2;
    const size_t smem = T2 * (8 + 2 * sizeof(E) + 4) + kStage * (4 + 2 * sizeof(E));
    const void *fn = (const void *)roll_kernel<E>;
    int grid = 0;
    int rc = launch_shape(fn, kBlock, smem, 0, g->num_sms, &grid);
    if (rc != KHOP_OK) return rc;
    if (grid_ctas > 0 && grid_ctas < grid) grid = grid_ctas;
    if ((uint64_t)grid > bs.part_rows) return KHOP_EINVAL;
    // counters, barrier word (the rolling state lives in `handoff`, `rdone`, `dirty`)
    cudaError_t e = cudaMemsetAsync(bs.ctl, 0, offsetof(CtlBlock, handoff), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&bs.ctl->bar, 0, sizeof(BarrierWords), st);
    if (e != cudaSuccess) return cuda_status(e);
    RollPlan p = plan;
    void *args[] = {(void *)&a, (void *)&p, (void *)&res};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, smem, st);
    return cuda_status(e);
}

}  // namespace

int roll_launch(khop_graph *g, BatchState &bs, const RollPlan &plan, RollResult *res, int grid_ctas,
                cudaStream_t st) {
    if (g->ewidth == 4) return roll_typed<uint32_t>(g, bs, plan, res, grid_ctas, st);
    return roll_typed<unsigned long long>(g, bs, plan, res, grid_ctas, st);
}

int batch_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                 uint64_t *out, cudaStream_t st, int lw) {
    if (lw == 4) {
        if (g->ewidth == 4) return launch_typed<uint32_t, 4>(g, seeds, ks, nq, out, st);
        return launch_typed<unsigned long long, 4>(g, seeds, ks, nq, out, st);
    }
    if (lw == 2) {
        if (g->ewidth == 4) return launch_typed<uint32_t, 2>(g, seeds, ks, nq, out, st);
        return launch_typed<unsigned long long, 2>(g, seeds, ks, nq, out, st);
    }
    if (g->ewidth == 4) return launch_typed<uint32_t, 1>(g, seeds, ks, nq, out, st);
    return launch_typed<unsigned long long, 1>(g, seeds, ks, nq, out, st);
}


}  // namespace khop
