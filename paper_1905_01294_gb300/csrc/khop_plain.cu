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

constexpr int kPushUnroll = 2;   // edges in flight per thread in a push tile
constexpr uint64_t kPrefetchEdges = 2048;    // next-query seed edges warmed into L2
constexpr uint32_t kSoloEdges = 2048;        // 1-hop queries with at most this many seed
                                             // out-edges run on one CTA
constexpr uint64_t kSoloRun = 8192;          // queries one CTA answers before the grid regroups
constexpr uint32_t kFuseDeg = 1024;          // seeds with at most this many out-edges get their
                                             // first two rounds fused into one grid round (every
                                             // CTA reads the seed row and its heads' offsets, so
                                             // a larger row makes the prelude L2-bound)
constexpr uint64_t kPrecheckEdges = 16384;   // push rounds this big (once over 1/32 of the
                                             // vertices are visited) read V before test-and-set
constexpr int kListWords = 16;   // bitmap words whose unvisited vertices a warp lists at once (pull)
constexpr int kFlatILP = 2;      // in-edges per lane per step of the flattened pull scan
constexpr int kListILP = 2;      // listed vertices per lane per step (their first in-edges in flight)
constexpr int kStage = 2048;     // queue items a CTA stages in shared memory per round
constexpr int kStagePosShift = 40;                       // staged count above, edges below
constexpr unsigned long long kStageEdgeMask = (1ull << kStagePosShift) - 1ull;

template <typename E>
struct PlainArgs {
    uint64_t n, nnz, n_noin;
    uint32_t nw;
    int symmetric;
    const E *rp;             // CSR row offsets [n+1]
    const uint32_t *ci;      // CSR heads [nnz]
    const E *cp;             // CSC column offsets [n+1]
    const uint32_t *ri;      // CSC tails [nnz]
    const uint32_t *noin;    // vertices without in-edges [nw]
    uint32_t *V0, *V1;       // visited bitmaps [nw]; queries alternate between them
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
    int keep_v;              // every query on the grid path (the visited bitmap is wanted)
    int32_t *levels;         // or null: levels[w] = r when round r discovers w
    uint64_t alpha_fx, beta_fx;   // Beamer's alpha and beta in 1/65536 units
    uint32_t tile_log2;
    uint32_t ebits;
    int stage;               // stage queue items per CTA (needs nnz < 2^40)
    uint64_t pull_cap;       // queue items a pull round writes (enough for a switch back to push)
    uint64_t timeout_ns;
    unsigned absent_at;      // testing: the last CTA skips its absent_at-th grid barrier (0 = never)
};

template <typename T>
__device__ __forceinline__ T sel3(T x0, T x1, T x2, unsigned i) {
    return i == 0 ? x0 : (i == 1 ? x1 : x2);
}

template <typename E>
struct Round {
    bool first, last;
    bool precheck;           // load the visited word before the test-and-set (big rounds)
    uint32_t seed;
    E seed_rs;               // row start of the seed (round 1)
    uint32_t *V;             // visited bitmap of this query
    const uint32_t *Fin;
    uint32_t *Fout;
    const E *Qpre_in, *Qrs_in;
    const uint32_t *TF_in;
    E *Qpre_out, *Qrs_out;
    uint32_t *TF_out;
    unsigned long long *qpack_out;
    uint64_t cap;            // queue items this round may write
    uint64_t items_in, mf;   // input frontier: queue items, out-edges
    bool solo;               // push round of one tile that fits the staging area: one CTA
                             // discovers everything, so its queue starts at 0 (no atomic)
    bool fused;              // rounds 1 and 2 in one: the items (the seed's distinct
                             // out-neighbours) are in shared memory, and heads in that
                             // set (or the seed) are skipped
    const uint32_t *nbr;     // fused: hash set of the seed's distinct out-neighbours
    uint32_t level;          // the round's number (its discoveries are at that hop distance)
    uint32_t rot;            // rotation of the push tiles over CTAs 1 .. G-1 (same in every CTA)
    uint32_t tl;             // log2 of the push tile (fused rounds: sized to the round)
};

// Per-CTA shared state of a round.
struct Shared {
    unsigned long long cnt;      // vertices discovered by the CTA
    unsigned long long scan;     // in-edges the CTA examined (pull)
    unsigned long long mf;       // out-edges of the vertices the CTA discovered
    unsigned long long stage;    // (staged items << 40) | staged out-edges
    unsigned long long limit;    // first staging position that did not fit (packed like stage)
    unsigned long long gbase;    // global (items << ebits | prefix) reserved for the staged items
    unsigned long long skipped;  // items not queued because the queue was past its cap
    int qfull;                   // this CTA saw the queue past its cap (pull rounds)
    unsigned long long slot[4];  // counters of the round just finished
    unsigned m1;                 // fused round: distinct out-neighbours of the seed
    unsigned pdeg;               // row length of the prelude held in the hash tables
    // the current query's result and stats, kept by thread 0 of CTA 0 only (in
    // registers they would be live in every thread across the whole round loop)
    unsigned long long q_count, q_te, q_bytes;
    unsigned q_rounds, q_pull;
    uint64_t ring_q;             // thread 0: the query whose ring_advance is due next
    int flag;
};

constexpr uint32_t kHashSlots = 4096;             // open addressing over <= 2048 keys
constexpr uint32_t kHashEmpty = 0xffffffffu;      // never a vertex id (n < 2^32)
static_assert(kHashSlots * 4 <= 3 * kStage * 4, "the one-CTA hash set lives in the staging area");

__device__ __forceinline__ uint32_t hash_home(uint32_t w) {
    return (w * 0x9E3779B1u) >> (32 - 12);   // 12 bits: kHashSlots = 4096
}

// Insert w; true if it was not in the set (slot = where it went).  Linear
// probing with CAS.
__device__ __forceinline__ bool hash_insert(uint32_t *tab, uint32_t w, uint32_t &slot) {
    uint32_t h = hash_home(w);
    for (;;) {
        const uint32_t old = atomicCAS(&tab[h], kHashEmpty, w);
        if (old == kHashEmpty) {
            slot = h;
            return true;
        }
        if (old == w) return false;
        h = (h + 1) & (kHashSlots - 1);
    }
}

// Insert w if absent; slot = where w is (inserted here or before).
__device__ __forceinline__ void hash_insert_at(uint32_t *tab, uint32_t w, uint32_t &slot) {
    uint32_t h = hash_home(w);
    for (;;) {
        const uint32_t old = atomicCAS(&tab[h], kHashEmpty, w);
        if (old == kHashEmpty || old == w) {
            slot = h;
            return;
        }
        h = (h + 1) & (kHashSlots - 1);
    }
}

// Is w in the set (no concurrent inserts)?
__device__ __forceinline__ bool hash_contains(const uint32_t *tab, uint32_t w) {
    uint32_t h = hash_home(w);
    for (;;) {
        const uint32_t x = tab[h];
        if (x == w) return true;
        if (x == kHashEmpty) return false;
        h = (h + 1) & (kHashSlots - 1);
    }
}

// Write queue item `pos` (out-edge prefix pre, row start rs, out-degree d)
// and point every push tile that begins inside its row at it.
template <typename E>
__device__ __forceinline__ void put_item(const PlainArgs<E> &a, const Round<E> &R, uint64_t pos,
                                         uint64_t pre, E rs, E d) {
    if (pos >= R.cap) return;
    R.Qpre_out[pos] = (E)pre;
    R.Qrs_out[pos] = rs;
    const uint64_t jf = (pre + (1ull << a.tile_log2) - 1ull) >> a.tile_log2;
    const uint64_t jl = (pre + (uint64_t)d - 1ull) >> a.tile_log2;
    for (uint64_t j = jf; j <= jl; ++j) R.TF_out[j] = (uint32_t)pos;
}

// Warp-collective bookkeeping of newly visited vertices.  `disc` marks a
// lane's new vertex w with row start rs and out-degree d.  Counts and
// out-edge sums go to CTA counters.  Unless this is the last round, vertices
// with out-edges join the next queue: the warp reserves consecutive slots in
// the CTA's shared staging area (one shared 64-bit atomic gives both the slot
// and the out-edge prefix), and the CTA publishes the whole area with one
// global atomic at the end of the round; a warp that finds the area full
// appends straight to the global queue.  set_f marks the vertex in the next
// frontier bitmap (push rounds; pull rounds store whole words).  Only vertices
// with out-edges need the bit: a pull round looks for parents, and a parent
// has an out-edge.
template <typename E>
__device__ __forceinline__ void record(const PlainArgs<E> &a, const Round<E> &R, bool disc,
                                       uint32_t w, E rs, E d, bool set_f, Shared &sh,
                                       E *st_pre, E *st_rs, E *st_d) {
    const unsigned m = __ballot_sync(FULL, disc);
    if (m == 0u) return;
    if (a.levels && disc) a.levels[w] = (int32_t)R.level;
    const int lane = threadIdx.x & 31;
    if (R.last) {
        if (lane == 0) atomicAdd(&sh.cnt, (unsigned long long)__popc(m));
        return;
    }
    const bool has = disc && d > 0;
    if (has && set_f) atomicOr(&R.Fout[w >> 5], 1u << (w & 31));
    const E dd = has ? d : (E)0;
    const E incl = warp_inclusive_sum(dd);
    const E tot = __shfl_sync(FULL, incl, 31);
    if (lane == 0) {
        atomicAdd(&sh.cnt, (unsigned long long)__popc(m));
        if (tot) atomicAdd(&sh.mf, (unsigned long long)tot);
    }
    const unsigned hm = __ballot_sync(FULL, has);
    if (hm == 0u) return;
    const int leader = __ffs(hm) - 1;
    const unsigned c = __popc(hm);
    const uint64_t rank = (uint64_t)__popc(hm & lanemask_lt());
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
        if (has) {
            const uint64_t p = (old >> kStagePosShift) + rank;
            st_pre[p] = (E)((old & kStageEdgeMask) + excl);
            st_rs[p] = rs;
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
        if (has)
            put_item(a, R, (old >> a.ebits) + rank, (old & ((1ull << a.ebits) - 1ull)) + excl, rs, d);
    }
}

// End of a round for one CTA: publish the staged queue items and flush the
// CTA counters.  Called by all threads of the CTA.
template <typename E, int BLOCK>
__device__ __forceinline__ void flush_round(const PlainArgs<E> &a, const Round<E> &R, Shared &sh,
                                            E *st_pre, E *st_rs, E *st_d,
                                            unsigned long long *slot_out) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long st = sh.stage;
        if (sh.limit < st) st = sh.limit;   // staged items are the prefix before the first miss
        const uint32_t nst = (uint32_t)(st >> kStagePosShift);
        if (nst) {
            const unsigned long long add = ((unsigned long long)nst << a.ebits) + (st & kStageEdgeMask);
            if (R.solo) {
                sh.gbase = 0ull;
                *R.qpack_out = add;
            } else {
                sh.gbase = atomicAdd(R.qpack_out, add);
            }
        }
        if (sh.skipped) atomicAdd(R.qpack_out, sh.skipped << a.ebits);
        sh.skipped = 0;
        sh.qfull = 0;
        if (sh.cnt) atomicAdd(slot_out + 1, sh.cnt);
        if (sh.scan) atomicAdd(slot_out + 2, sh.scan);
        if (sh.mf) atomicAdd(slot_out + 3, sh.mf);
        sh.cnt = sh.scan = sh.mf = 0;
        sh.stage = 0;
        sh.limit = ~0ull;
        sh.flag = (int)nst;
    }
    __syncthreads();
    const uint32_t nst = (uint32_t)sh.flag;
    if (nst) {
        const uint64_t gpos = sh.gbase >> a.ebits;
        const uint64_t gpre = sh.gbase & ((1ull << a.ebits) - 1ull);
        for (uint32_t t = threadIdx.x; t < nst; t += BLOCK)
            put_item(a, R, gpos + t, gpre + (uint64_t)st_pre[t], st_rs[t], st_d[t]);
    }
}

// Push round: tiles of T consecutive frontier out-edges, one CTA per tile.
template <typename E, int BLOCK>
__device__ __forceinline__ void push_round(const PlainArgs<E> &a, const Round<E> &R, E *s_pre,
                                           E *s_rs, Shared &sh, E *st_pre, E *st_rs, E *st_d) {
    const uint32_t tl = R.tl;
    const uint64_t T = 1ull << tl;
    const uint64_t ntiles = (R.mf + T - 1) >> tl;
    // CTA 0 writes the query results between queries: it takes tile G - 1.
    // CTAs 1 .. G-1 take tiles 0 .. G-2 in an order rotated every round, so
    // the few tiles of a small round go to CTAs other than the previous
    // round's workers (which arrive last at its barrier and list the next
    // query's prelude only then).
    const uint32_t g1 = gridDim.x - 1u;
    uint32_t rk = blockIdx.x - 1u + R.rot;   // R.rot < max(g1, 1)
    if (rk >= g1) rk -= g1;
    const uint64_t rank = blockIdx.x == 0 ? (uint64_t)g1 : (uint64_t)rk;
    for (uint64_t j = rank; j < ntiles; j += gridDim.x) {
        const uint64_t e0 = j << tl;
        const uint64_t e1 = min(e0 + T, R.mf);
        uint32_t nitems;
        uint32_t hint = 0;
        if (R.fused) {
            // all items are in shared memory already: start at the tile's first
            nitems = (uint32_t)R.items_in;
            uint32_t lo = 0, hi = nitems - 1;   // largest item with prefix <= e0
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if ((uint64_t)s_pre[mid] <= e0) lo = mid; else hi = mid - 1;
            }
            hint = lo;
        } else if (R.first) {
            if (threadIdx.x == 0) {
                s_pre[0] = (E)0;
                s_rs[0] = R.seed_rs;
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
        if (!R.fused) __syncthreads();
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
                E rs = 0, re = 0;
                // Round 1: every distinct neighbour of the seed is new, so its
                // row offsets are loaded alongside the test-and-set.
                const bool early = R.first && !R.last && ok[u];
                if (early) {
                    rs = a.rp[w[u]];
                    re = a.rp[w[u] + 1];
                }
                // fused round: the seed and its out-neighbours belong to round 0/1
                const bool go = ok[u] && !(R.fused && (w[u] == R.seed || hash_contains(R.nbr, w[u])));
                if (go) {
                    const uint32_t wi = w[u] >> 5, bit = 1u << (w[u] & 31);
                    if (!R.precheck || !(R.V[wi] & bit)) disc = !(atomicOr(&R.V[wi], bit) & bit);
                }
                E d = 0;
                if (disc && !R.last) {
                    if (!early) {
                        rs = a.rp[w[u]];
                        re = a.rp[w[u] + 1];
                    }
                    d = re - rs;
                }
                record(a, R, disc, w[u], rs, d, true, sh, st_pre, st_rs, st_d);
            }
        }
        if (!R.fused) __syncthreads();
    }
}

// Prelude of a fused first round, run by every CTA on its own: the seed's
// distinct out-neighbours other than the seed (q_1 of the paper's iteration,
// Sec. III) into the shared hash set `tab`, in the order of their first
// position in the seed's row (the same order in every CTA, so all CTAs cut
// round 2's edge list the same way), their row starts into s_rs and their
// out-edge prefix sums into s_pre (s_pre[m1] = m_f of round 2).  `pos` holds
// each key's first position.  The row offsets of every position are loaded
// alongside the inserts (a repeated head just loads its row twice), and one
// scan over the threads -- which hold consecutive positions -- gives both each
// kept head's index and its prefix.  `pslot` records the slot of every row
// position and sh.pdeg the row length, so prelude_clear empties only those
// slots.  Returns m1 (the caller empties the tables after the round).
template <typename E, int BLOCK>
__device__ __forceinline__ uint32_t fused_prelude(const PlainArgs<E> &a, uint32_t s, E rs0,
                                                  uint32_t deg, uint32_t *tab, uint32_t *pos, uint16_t *pslot,
                                                  E *s_pre, E *s_rs, Shared &sh) {
    constexpr int kPer = (int)(kFuseDeg / BLOCK);
    constexpr uint32_t kWarpPos = 32u * (uint32_t)kPer;   // row positions a warp holds
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ unsigned long long s_wtot[32];   // per warp: kept count << 40 | edge sum
    // thread t holds row positions t * kPer .. t * kPer + kPer - 1; warps whose
    // positions all lie past the row's end only join the barriers
    const uint32_t na = (deg + kWarpPos - 1u) / kWarpPos;
    const bool active = (uint32_t)warp < na;
    uint32_t w[kPer], slot[kPer];
    E rsv[kPer], rev[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        w[u] = kHashEmpty;
        slot[u] = kHashSlots;
        rsv[u] = 0;
        rev[u] = 0;
    }
    if (active) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const uint32_t e = threadIdx.x * kPer + u;
            if (e < deg) w[u] = a.ci[(uint64_t)rs0 + e];
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            if (w[u] != kHashEmpty) {
                rsv[u] = a.rp[w[u]];
                rev[u] = a.rp[w[u] + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            if (w[u] != kHashEmpty && w[u] != s) {
                hash_insert_at(tab, w[u], slot[u]);
                atomicMin(&pos[slot[u]], threadIdx.x * kPer + u);
            }
            if (threadIdx.x * kPer + u < deg) pslot[threadIdx.x * kPer + u] = (uint16_t)slot[u];
        }
    }
    if (threadIdx.x == 0) sh.pdeg = deg;
    __syncthreads();
    // keep each neighbour at its first position: (count, edges) of this thread
    unsigned keep = 0;
    unsigned long long mine = 0, incl = 0;
    if (active) {
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (slot[u] < kHashSlots && pos[slot[u]] == threadIdx.x * kPer + u) {
                keep |= 1u << u;
                mine += (1ull << 40) + (unsigned long long)(rev[u] - rsv[u]);
            }
        incl = warp_inclusive_sum(mine);
        if (lane == 31) s_wtot[warp] = incl;
    }
    __syncthreads();
    if (warp == 0) {   // inclusive scan of the active warps' totals
        unsigned long long x = (uint32_t)lane < na ? s_wtot[lane] : 0ull;
        x = warp_inclusive_sum(x);
        if ((uint32_t)lane < na) s_wtot[lane] = x;
    }
    __syncthreads();
    const unsigned long long tot = na ? s_wtot[na - 1u] : 0ull;
    if (active) {
        const unsigned long long base = incl - mine + (warp ? s_wtot[warp - 1] : 0ull);
        uint32_t idx = (uint32_t)(base >> 40);
        E pre = (E)(base & ((1ull << 40) - 1ull));
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if ((keep >> u) & 1u) {
                s_pre[idx] = pre;
                s_rs[idx] = rsv[u];
                pre += rev[u] - rsv[u];
                ++idx;
            }
    }
    const uint32_t m1 = (uint32_t)(tot >> 40);
    if (threadIdx.x == 0) s_pre[m1] = (E)(tot & ((1ull << 40) - 1ull));
    __syncthreads();
    return m1;
}

// Empty the prelude's hash set and first-position table: only the slots its
// row positions filled (a repeated head empties its slot twice).
template <int BLOCK>
__device__ __forceinline__ void prelude_clear(uint32_t *tab, uint32_t *pos, const uint16_t *pslot,
                                              const Shared &sh) {
    const uint32_t deg = sh.pdeg;
    for (uint32_t p = threadIdx.x; p < deg; p += BLOCK) {
        const uint32_t sl = pslot[p];
        if (sl < kHashSlots) {
            tab[sl] = kHashEmpty;
            pos[sl] = 0xffffffffu;
        }
    }
}

// Pull round (masked SpMV over the unvisited vertices).  Warps take groups
// of kListWords consecutive bitmap words (one per lane, grid-strided) and
// list the group's unvisited vertices with in-edges -- V OR the in-edge-less
// bitmap, complemented -- by a warp scan of the words' popcounts; the list is
// then worked 32 vertices at a time, one per lane (its word by a shuffle
// search over the scan, its bit by __fns; kListILP vertices per lane, their
// first in-edges in flight together), so every lane has a vertex
// whether the unvisited vertices are dense (early rounds) or one or two per
// word (late rounds of a deep query).  Each vertex first checks its first two
// in-edges against the frontier bitmap; the in-edges of the vertices still
// unresolved are then scanned as one flattened list: the warp takes the next
// 32 * kFlatILP edges of the concatenated remaining in-edge lists (a
// load-balanced search over the lanes' remaining counts), and a vertex drops
// out as soon as one of its in-neighbours is in the frontier.  Found
// vertices are marked in V and F_out with one reduction per bitmap word (F_out
// was zeroed one round ahead).
template <typename E, int BLOCK>
__device__ __forceinline__ void pull_round(const PlainArgs<E> &a, const Round<E> &R, Shared &sh,
                                           E *s_winc, E *s_wpos, E *st_pre, E *st_rs, E *st_d) {
    const int lane = threadIdx.x & 31;
    E *winc = s_winc + (threadIdx.x >> 5) * 32;
    E *wpos = s_wpos + (threadIdx.x >> 5) * 32;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * BLOCK) >> 5;
    const uint32_t tail_open = (a.n & 31) ? ~(~0u << (a.n & 31)) : ~0u;   // valid bits of the last word
    uint64_t scanned = 0;
    for (uint64_t c0 = gwarp * kListWords; c0 < a.nw; c0 += nwarps * kListWords) {
        const uint64_t il = c0 + (uint64_t)lane;
        uint32_t wl = ~0u;
        if (lane < kListWords && il < a.nw) {
            wl = R.V[il] | a.noin[il];
            if (il == a.nw - 1) wl |= ~tail_open;
        }
        const uint32_t fr = ~wl;   // this lane's word: unvisited vertices with in-edges
        const uint32_t cnt = (uint32_t)__popc(fr);
        const uint32_t incl = warp_inclusive_sum(cnt);
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        for (uint32_t base = 0; base < total; base += 32 * kListILP) {
            // lane l takes list positions base + j * 32 + l (j < kListILP): their
            // first in-edges are loaded and checked together
            uint64_t v[kListILP];
            E b[kListILP], e[kListILP], pos[kListILP];
            bool unv[kListILP], found[kListILP];
#pragma unroll
            for (int j = 0; j < kListILP; ++j) {
                const uint32_t x = base + (uint32_t)(j * 32 + lane);
                int L = 0;                                   // first lane whose inclusive count exceeds x
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t im = __shfl_sync(FULL, incl, L + step - 1);
                    if (im <= x) L += step;
                }
                unv[j] = x < total;
                L = min(L, 31);
                const uint32_t fro = __shfl_sync(FULL, fr, L);
                const uint32_t exo = __shfl_sync(FULL, incl - cnt, L);
                const uint32_t bit = unv[j] ? __fns(fro, 0u, (int)(x - exo) + 1) : 0u;
                v[j] = ((c0 + (uint64_t)L) << 5) + (uint64_t)bit;
                b[j] = 0;
                e[j] = 0;
                if (unv[j]) {
                    b[j] = a.cp[v[j]];
                    e[j] = a.cp[v[j] + 1];
                }
                pos[j] = b[j];
            }
            uint32_t u0[kListILP], u1[kListILP];
            bool l0[kListILP], l1[kListILP];
#pragma unroll
            for (int j = 0; j < kListILP; ++j) {
                l0[j] = unv[j] && pos[j] < e[j];
                l1[j] = l0[j] && pos[j] + 1 < e[j];
                u0[j] = l0[j] ? a.ri[pos[j]] : 0u;
                u1[j] = l1[j] ? a.ri[pos[j] + 1] : 0u;
            }
#pragma unroll
            for (int j = 0; j < kListILP; ++j) {
                bool f = l0[j] && ((R.Fin[u0[j] >> 5] >> (u0[j] & 31)) & 1u);
                f = f || (l1[j] && ((R.Fin[u1[j] >> 5] >> (u1[j] & 31)) & 1u));
                found[j] = f;
                pos[j] += (E)l0[j] + (E)l1[j];
                scanned += (uint64_t)l0[j] + (uint64_t)l1[j];
            }
#pragma unroll
            for (int j = 0; j < kListILP; ++j) {
                E rem = (unv[j] && !found[j]) ? e[j] - pos[j] : (E)0;
                while (__any_sync(FULL, rem > 0)) {
                    const E inc2 = warp_inclusive_sum(rem);
                    const E tot2 = __shfl_sync(FULL, inc2, 31);
                    const E exc2 = inc2 - rem;
                    winc[lane] = inc2;
                    wpos[lane] = pos[j] - exc2;
                    __syncwarp();
                    const uint32_t chunk = (uint32_t)min(tot2, (E)(32 * kFlatILP));
                    unsigned hits = 0;
#pragma unroll
                    for (int t = 0; t < kFlatILP; ++t) {
                        const uint32_t xx = (uint32_t)(t * 32 + lane);
                        if (xx < chunk) {
                            int lo = 0, hi = 31;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (winc[mid] > (E)xx) hi = mid; else lo = mid + 1;
                            }
                            const uint32_t uu = a.ri[wpos[lo] + (E)xx];
                            if ((R.Fin[uu >> 5] >> (uu & 31)) & 1u) hits |= 1u << lo;
                        }
                    }
                    hits = __reduce_or_sync(FULL, hits);
                    const E consumed = (E)chunk > exc2 ? min(rem, (E)chunk - exc2) : (E)0;
                    pos[j] += consumed;
                    rem -= consumed;
                    if ((hits >> lane) & 1u) {
                        found[j] = true;
                        rem = 0;
                    }
                    if (lane == 0) scanned += chunk;
                    __syncwarp();
                }
            }
#pragma unroll
            for (int j = 0; j < kListILP; ++j) {
                // The list runs in vertex order, so lanes holding the same word
                // are consecutive: a segmented OR-scan gives the last lane of
                // each run the run's found bits, and it alone marks them in V
                // and F_out.
                {
                    const uint32_t wv = unv[j] ? (uint32_t)(v[j] >> 5) : 0xffffffffu;
                    uint32_t acc = found[j] ? 1u << (v[j] & 31) : 0u;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL, acc, o);
                        const uint32_t yw = __shfl_up_sync(FULL, wv, o);
                        if (lane >= o && yw == wv) acc |= y;
                    }
                    const uint32_t nw = __shfl_down_sync(FULL, wv, 1);
                    if (acc && (lane == 31 || nw != wv)) {
                        atomicOr(&R.V[wv], acc);
                        if (!R.last) atomicOr(&R.Fout[wv], acc);
                    }
                }
                E rs = 0, d = 0;
                if (found[j] && !R.last) {
                    if (a.symmetric) { rs = b[j]; d = e[j] - b[j]; }
                    else { rs = a.rp[v[j]]; d = a.rp[v[j] + 1] - rs; }
                }
                record(a, R, found[j], (uint32_t)v[j], rs, d, false, sh, st_pre, st_rs, st_d);
            }
        }
    }
    scanned = warp_sum(scanned);
    if (lane == 0 && scanned) atomicAdd(&sh.scan, (unsigned long long)scanned);
}

// A query that needs a traversal: its seed, k and seed row.
template <typename E>
struct QueryHead {
    uint32_t s, k;
    E rs, re;
};

// Answer the queries that need no traversal -- k = 0, a seed >= n, or a seed
// without out-edges (count 0 and TE 0) -- and return the index of the next
// query that does, with its head in *h.  Only thread 0 of CTA 0 writes (when
// `write` is set).
template <typename E>
__device__ __forceinline__ uint64_t skip_trivial(const PlainArgs<E> &a, uint64_t q, bool write,
                                                 uint64_t &t_prev, QueryHead<E> *h) {
    for (; q < a.nq; ++q) {
        const uint32_t s = a.seeds[q];
        const uint32_t k = a.ks ? a.ks[q] : a.k_all;
        if (s < a.n && k > 0) {
            const E rs = a.rp[s], re = a.rp[s + 1];
            if (re > rs) {
                if (h) *h = QueryHead<E>{s, k, rs, re};
                break;
            }
        }
        if (write) {
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

// Visited bitmap for the next query: just its seed (stores only).  Pull
// rounds treat the vertices without in-edges as visited too -- no round can
// reach them -- by OR-ing in that bitmap as they read V.  Grid-stride over the
// words.
template <typename E>
__device__ __forceinline__ void prep_visited(const PlainArgs<E> &a, uint32_t *V, bool any,
                                             uint32_t seed, uint64_t gtid, uint64_t gthreads) {
    const uint64_t sw = any ? (uint64_t)(seed >> 5) : ~0ull;
    const uint32_t sb = 1u << (seed & 31);
    for (uint64_t i = gtid; i < a.nw; i += gthreads) V[i] = i == sw ? sb : 0u;
}

// Look-ahead over the query list: the heads of the next queries, fetched by
// thread 0 of each CTA with asynchronous copies into a shared-memory ring, so
// no thread waits on the dependent loads seeds[i] -> rp[seed].  Each
// query start commits two copy groups -- the row bounds of q + 4 and the seed
// and k of q + 6 -- and waits only for the groups of two query starts ago, so
// every copy has two queries' time to land.  After ring_advance(q) the heads
// of q + 1 and q + 2 are complete; once published, other warps prefetch the
// row of q + 2 into L2.
template <typename E>
struct Peek {
    uint32_t s, k;
    E rs, re;
};
constexpr int kRing = 8;

template <typename E>
__device__ __forceinline__ void ring_stage1(const PlainArgs<E> &a, Peek<E> *ring, uint64_t i) {
    Peek<E> &p = ring[i % kRing];
    if (i < a.nq) {
        cp_async<4>(&p.s, a.seeds + i);
        if (a.ks) cp_async<4>(&p.k, a.ks + i);
        else p.k = a.k_all;
    } else {
        p.s = 0xffffffffu;
        p.k = 0u;
    }
    cp_async_commit();
}

template <typename E>
__device__ __forceinline__ void ring_stage2(const PlainArgs<E> &a, Peek<E> *ring, uint64_t i) {
    Peek<E> &p = ring[i % kRing];
    const uint32_t s = p.s;
    if (i < a.nq && s < a.n) {
        cp_async<(int)sizeof(E)>(&p.rs, a.rp + s);
        cp_async<(int)sizeof(E)>(&p.re, a.rp + s + 1);
    } else {
        p.rs = (E)0;
        p.re = (E)0;
    }
    cp_async_commit();
}

// Warm L2 with the row of query i (at most kSoloEdges out-edges; its head must
// be complete and published): thread t of nt takes every nt-th 128-byte line.
template <typename E>
__device__ __forceinline__ void ring_prefetch_row(const PlainArgs<E> &a, const Peek<E> *ring, uint64_t i,
                                                  unsigned t, unsigned nt) {
    const Peek<E> &p = ring[i % kRing];
    if (i < a.nq && p.s < a.n && p.re > p.rs) {
        const uint64_t nd = min((uint64_t)(p.re - p.rs), (uint64_t)kSoloEdges);
        constexpr uint64_t kLine = 128 / sizeof(uint32_t);
        for (uint64_t e = (uint64_t)t * kLine; e < nd; e += (uint64_t)nt * kLine)
            prefetch_l2(a.ci + (uint64_t)p.rs + e);
    }
}

// Thread 0, when query q starts.
template <typename E>
__device__ __forceinline__ void ring_advance(const PlainArgs<E> &a, Peek<E> *ring, uint64_t q) {
    cp_async_wait_group<2>();   // the groups of ring_advance(q - 2) and before
    ring_stage2(a, ring, q + 4);
    ring_stage1(a, ring, q + 6);
}

// Thread 0: (re)start the ring in the state ring_advance(q) expects: heads of
// q + 1 .. q + 3 complete, seeds of q + 4, q + 5 in place (nothing pending).
template <typename E>
__device__ __forceinline__ void ring_restart(const PlainArgs<E> &a, Peek<E> *ring, uint64_t q) {
    cp_async_wait_all();
    for (uint64_t i = q + 1; i <= q + 5; ++i) ring_stage1(a, ring, i);
    cp_async_wait_all();
    for (uint64_t i = q + 1; i <= q + 3; ++i) ring_stage2(a, ring, i);
    cp_async_wait_all();
    ring_prefetch_row(a, ring, q + 1, 0u, 1u);
}

// The first query after q that needs a traversal (no writes), from the ring's
// head of q + 1 (complete and published since query q started); scans on
// only when q + 1 needs no traversal.
template <typename E>
__device__ __forceinline__ uint64_t ring_next(const PlainArgs<E> &a, const Peek<E> *ring, uint64_t q,
                                              QueryHead<E> &h) {
    if (q + 1 >= a.nq) return a.nq;
    const Peek<E> &p = ring[(q + 1) % kRing];
    if (p.s < a.n && p.k > 0 && p.re > p.rs) {
        h = QueryHead<E>{p.s, p.k, p.rs, p.re};
        return q + 1;
    }
    uint64_t t_dummy = 0;
    return skip_trivial(a, q + 1, false, t_dummy, &h);
}

// A query that one CTA answers alone: k = 1 and at most kSoloEdges out-edges
// at the seed.  Its single round is q_1 = A^T e_s minus the seed, so its
// count is the number of distinct out-neighbours of s other than s: one CTA
// finds them with a hash set in shared memory -- no visited bitmap, no
// frontier, no grid barrier -- while the other CTAs wait at one barrier for
// the whole run of such queries.  (Pull-only mode keeps the grid path.)
template <typename E>
__device__ __forceinline__ bool solo_query(const QueryHead<E> &h, bool all_pull) {
    return !all_pull && h.k == 1 && (uint64_t)(h.re - h.rs) <= (uint64_t)kSoloEdges;
}

static_assert(kHashSlots == 2 * kSoloEdges, "load factor <= 1/2");

// Answer 1-hop queries from query q on, on this CTA only, until the next one
// is not such a query (or kSoloRun were answered or the list ends).  The
// visited bitmap V is not used: on entry it holds the seed of query q, on
// return the seed of the query the grid goes on with.  On return q and cur
// name that query and thread 0 has left (q, head) in ctl->handoff for the
// other CTAs.  Thread 0 writes the results (it is b0) and keeps the
// look-ahead ring.
template <typename E, int BLOCK>
__device__ __noinline__ void solo_run(const PlainArgs<E> &args, uint32_t *V, uint64_t &q,
                                      QueryHead<E> &cur, uint64_t &t_prev, Shared &sh,
                                      Peek<E> *ring, uint32_t *tab) {
    // A private copy: its fields stay in registers (the launch arguments seen
    // through a reference would be reloaded after every store and copy).
    const PlainArgs<E> a = args;
    constexpr int kPer = (int)(kSoloEdges / BLOCK);
    const int lane = threadIdx.x & 31;
    const uint32_t s_first = cur.s;
    for (uint32_t i = threadIdx.x; i < kHashSlots; i += BLOCK) tab[i] = kHashEmpty;
    if (threadIdx.x == 0 && sh.ring_q != q) ring_restart(a, ring, q);   // else still in step
    // the seed row of each query is loaded one query ahead (below), so its
    // latency overlaps the previous query's bookkeeping
    uint32_t w[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const uint32_t e = (uint32_t)(u * BLOCK) + threadIdx.x;
        w[u] = e < (uint32_t)(cur.re - cur.rs) ? a.ci[(uint64_t)cur.rs + e] : kHashEmpty;
    }
    __syncthreads();
    for (uint64_t run = 1;; ++run) {
        if (threadIdx.x == 0) ring_advance(a, ring, q);
        const uint32_t deg = (uint32_t)(cur.re - cur.rs);
        uint32_t slot[kPer];
        unsigned c = 0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            slot[u] = kHashSlots;
            if ((uint32_t)(u * BLOCK) >= deg) break;   // uniform over the CTA
            const bool disc = w[u] != kHashEmpty && w[u] != cur.s && hash_insert(tab, w[u], slot[u]);
            c += (unsigned)__popc(__ballot_sync(FULL, disc));
        }
        if (lane == 0 && c) atomicAdd(&sh.cnt, (unsigned long long)c);
        __syncthreads();   // counts complete; the ring's heads of q + 1, q + 2 published
        QueryHead<E> nxt{0u, 0u, (E)0, (E)0};
        const uint64_t qn = ring_next(a, ring, q, nxt);
        if (qn < a.nq && solo_query(nxt, false)) {   // the next query's seed row, in flight from here
            const uint32_t dn = (uint32_t)(nxt.re - nxt.rs);
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint32_t e = (uint32_t)(u * BLOCK) + threadIdx.x;
                w[u] = e < dn ? a.ci[(uint64_t)nxt.rs + e] : kHashEmpty;
            }
        }
        if (threadIdx.x >= 32) ring_prefetch_row(a, ring, q + 2, threadIdx.x - 32u, BLOCK - 32u);
        if (threadIdx.x == 0) {
            const uint64_t cnt = sh.cnt;
            sh.cnt = 0;
            const uint64_t now = globaltimer_ns();
            a.out[q] = cnt;
            if (a.out_te) a.out_te[q] = deg;
            if (a.stats) {
                khop_query_stats st{t_prev, now, (uint64_t)deg, 4ull * deg + 2ull * sizeof(E) + 4ull, 1u, 0u};
                a.stats[q] = st;
            }
            if (a.per_hop) {
                for (uint32_t r = 0; r < a.hop_stride; ++r)
                    a.per_hop[q * a.hop_stride + r] = r == 0 ? 1ull : (r == 1 ? cnt : 0ull);
            }
            t_prev = now;
            if (qn > q + 1) {   // answer the trivial queries up to qn; restart the look-ahead
                skip_trivial(a, q + 1, true, t_prev, (QueryHead<E> *)nullptr);
                if (qn < a.nq) ring_restart(a, ring, qn);
            }
        }
        // empty the slots this query filled
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (slot[u] < kHashSlots) tab[slot[u]] = kHashEmpty;
        q = qn;
        cur = nxt;
        if (q >= a.nq || !solo_query(cur, false) || run >= kSoloRun) break;
        __syncthreads();   // the set is empty again before the next query's inserts
    }
    if (threadIdx.x == 0) {
        sh.ring_q = q;   // ready for q (its copies may still be in flight)
        // V for the grid's next query: its seed only
        V[s_first >> 5] = 0u;
        if (q < a.nq) V[cur.s >> 5] = 1u << (cur.s & 31);
        a.ctl->handoff[0] = q;
        a.ctl->handoff[1] = (unsigned long long)cur.s | ((unsigned long long)cur.k << 32);
        a.ctl->handoff[2] = (unsigned long long)cur.rs;
        a.ctl->handoff[3] = (unsigned long long)cur.re;
    }
}

template <typename E, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) plain_kernel(const PlainArgs<E> a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const uint32_t tcap = max(1u << a.tile_log2, kFuseDeg) + 2u;
    E *s_pre = (E *)dyn_smem;                         // push tile items [max(T, fused) + 2]
    E *s_rs = s_pre + tcap;
    E *st_pre = s_rs + tcap;                          // staged queue items [kStage]
    E *st_rs = st_pre + kStage;
    E *st_d = st_rs + kStage;
    uint32_t *s_nbr = (uint32_t *)(st_d + kStage);    // fused rounds: hash set [kHashSlots]
    uint32_t *s_npos = s_nbr + kHashSlots;            //   and each key's first row position
    uint16_t *s_pslot = (uint16_t *)(s_npos + kHashSlots);   //   and each row position's slot [kFuseDeg]
    __shared__ Shared sh;
    __shared__ E s_winc[BLOCK], s_wpos[BLOCK];        // flattened pull scan, 32 per warp
    __shared__ Peek<E> s_ring[kRing];                 // look-ahead over the query list

    const bool b0 = blockIdx.x == 0 && threadIdx.x == 0;
    const uint64_t gtid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * BLOCK;
    if (threadIdx.x == 0) {
        sh.cnt = sh.scan = sh.mf = sh.stage = 0;
        sh.limit = ~0ull;
        sh.skipped = 0;
        sh.qfull = 0;
        sh.pdeg = 0;
    }
    uint64_t t_prev = b0 ? globaltimer_ns() : 0;
    BarState bsense = barrier_start(&a.ctl->bar, a.absent_at);
    if (threadIdx.x == 0) sh.ring_q = ~0ull;
    for (uint32_t i = threadIdx.x; i < kHashSlots; i += BLOCK) {
        s_nbr[i] = kHashEmpty;
        s_npos[i] = 0xffffffffu;
    }
    __syncthreads();

    const bool all_pull = a.direction == KHOP_DIR_PULL;
    unsigned long long *slots = (unsigned long long *)a.ctl->slot;

    // Launch prologue: frontier bitmaps zero, V0 = {first seed}.
    QueryHead<E> cur{0u, 0u, (E)0, (E)0}, nxt{0u, 0u, (E)0, (E)0};
    uint64_t q = skip_trivial(a, 0, b0, t_prev, &cur);
    for (uint64_t i = gtid; i < a.nw; i += gthreads) {
        a.F0[i] = 0u;
        a.F1[i] = 0u;
        a.F2[i] = 0u;
    }
    prep_visited(a, a.V0, q < a.nq, cur.s, gtid, gthreads);
    if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns)) return;

    uint64_t rdone = 0;   // rounds run in this launch (selects the rotating buffers)
    uint32_t rot = 0;     // push tile rotation (see push_round)
    unsigned par = 0;     // which visited bitmap the current query uses
    bool pre_have = false;   // the current query's fused prelude already ran
    uint32_t pre_m1 = 0;     //   (at the previous query's last barrier) and its m1
    while (q < a.nq) {
        if (!a.keep_v && solo_query(cur, all_pull)) {
            if (blockIdx.x == 0)
                solo_run<E, BLOCK>(a, par ? a.V1 : a.V0, q, cur, t_prev, sh, s_ring, (uint32_t *)st_pre);
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, a.ctl->handoff, sh.slot, 4,
                              a.timeout_ns))
                return;
            q = sh.slot[0];
            cur.s = (uint32_t)sh.slot[1];
            cur.k = (uint32_t)(sh.slot[1] >> 32);
            cur.rs = (E)sh.slot[2];
            cur.re = (E)sh.slot[3];
            continue;
        }
        const uint32_t s = cur.s;
        const uint32_t k = cur.k;
        uint32_t *V = par ? a.V1 : a.V0;
        uint32_t *Vnext = par ? a.V0 : a.V1;
        // The next query from the look-ahead ring (no wait on its loads).
        if (threadIdx.x == 0) {
            if (sh.ring_q != q) ring_restart(a, s_ring, q);
            ring_advance(a, s_ring, q);
            sh.ring_q = q + 1;
        }
        __syncthreads();
        const uint64_t qn = ring_next(a, s_ring, q, nxt);
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x >= 32)
            ring_prefetch_row(a, s_ring, q + 2, threadIdx.x - 32u, BLOCK - 32u);
        if (all_pull) {
            // Round 1 pulls from the bitmap {s}: set it up before the round.
            uint32_t *Fs = sel3(a.F0, a.F1, a.F2, (unsigned)(rdone % 3));
            const uint64_t sw = s >> 5;
            for (uint64_t i = gtid; i < a.nw; i += gthreads) Fs[i] = i == sw ? 1u << (s & 31) : 0u;
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, nullptr, nullptr, 0, a.timeout_ns))
                return;
        }
        uint64_t mf = (uint64_t)(cur.re - cur.rs);   // out-edges of the frontier {s}
        uint64_t items = 1;
        uint64_t nf = 1;
        uint64_t sum_mf = 0, visited = 1;
        if (b0) {
            sh.q_count = sh.q_te = sh.q_bytes = 0ull;
            sh.q_rounds = sh.q_pull = 0u;
        }
        int prev = DIR_PUSH;
        for (uint32_t r = 1; r <= k && mf > 0; ++r) {
            ++rdone;
            rot += 7u;   // the tile rotation of this round, below max(G - 1, 1)
            while (rot >= max(gridDim.x - 1u, 1u)) rot -= max(gridDim.x - 1u, 1u);
            const unsigned iin = (unsigned)((rdone - 1) % 3), iout = (unsigned)(rdone % 3);
            const unsigned izero = (unsigned)((rdone + 1) % 3);
            const unsigned qin = (unsigned)((rdone - 1) & 1), qout = (unsigned)(rdone & 1);
            int dir;
            if (r == 1) dir = all_pull ? DIR_PULL : DIR_PUSH;
            else if (a.direction == KHOP_DIR_PUSH) dir = DIR_PUSH;
            else if (all_pull) dir = DIR_PULL;
            else {
                const uint64_t mu = a.nnz - (sum_mf + mf);   // out-edges of unvisited vertices
                if (prev == DIR_PUSH)
                    dir = fx_gt(mf, a.alpha_fx, mu) ? DIR_PULL : DIR_PUSH;
                else
                    dir = (fx_lt(nf, a.beta_fx, a.n) && items <= a.pull_cap)
                              ? DIR_PUSH : DIR_PULL;
            }
            // Zero what round r+1 writes (last read in round r-1).
            uint32_t *Fz = sel3(a.F0, a.F1, a.F2, izero);
            for (uint64_t i = gtid; i < a.nw; i += gthreads) Fz[i] = 0u;
            if (b0) {
                slots[kSlotWords * izero + 0] = 0ull;
                slots[kSlotWords * izero + 1] = 0ull;
                slots[kSlotWords * izero + 2] = 0ull;
                slots[kSlotWords * izero + 3] = 0ull;
                slots[kSlotWords * izero + 4] = 0ull;
            }
            if (b0) sh.q_te += mf;
            // Rounds 1 and 2 in one grid round (k >= 2, a push from a small seed
            // row): every CTA lists q_1 itself, so round 1 needs no barrier.
            // Not when Beamer's test would pull in round 2.
            uint32_t m1 = 0;
            uint64_t mf2 = 0;
            bool fused = false;
            if (r == 1 && k >= 2 && !all_pull && a.stage && mf <= (uint64_t)kFuseDeg) {
                m1 = pre_have ? pre_m1
                              : fused_prelude<E, BLOCK>(a, s, cur.rs, (uint32_t)mf, s_nbr, s_npos, s_pslot, s_pre,
                                                        s_rs, sh);
                pre_have = false;
                mf2 = (uint64_t)s_pre[m1];
                const uint64_t mu = a.nnz - (mf + mf2);
                fused = a.direction == KHOP_DIR_PUSH || !fx_gt(mf2, a.alpha_fx, mu);
                if (fused && blockIdx.x == 0)   // q_1 visited (round 2 skips it)
                    for (uint32_t p = threadIdx.x; p < sh.pdeg; p += BLOCK) {
                        const uint32_t sl = s_pslot[p];
                        if (sl < kHashSlots) {
                            const uint32_t x = s_nbr[sl];
                            atomicOr(&V[x >> 5], 1u << (x & 31));
                            if (a.levels) a.levels[x] = 1;
                        }
                    }
                if (!fused) {
                    prelude_clear<BLOCK>(s_nbr, s_npos, s_pslot, sh);
                    __syncthreads();
                }
            }
            Round<E> R;
            R.first = r == 1 && !fused;
            R.last = r + (fused ? 1u : 0u) == k;
            R.precheck = mf > kPrecheckEdges && visited * 32 > a.n;
            R.fused = fused;
            R.nbr = s_nbr;
            R.level = fused ? 2u : r;
            R.rot = rot;
            // A fused round's items are in every CTA's shared memory, so its
            // tiles need no tile map: they grow to about m_f / G edges, so
            // that each CTA's passes of BLOCK * kPushUnroll edges run full
            // (fixed tiles of T < BLOCK * kPushUnroll leave slots empty).
            R.tl = a.tile_log2;
            if (fused)
                while (R.tl < 24u && ((uint64_t)gridDim.x << R.tl) < mf2) ++R.tl;
            R.seed = s;
            R.seed_rs = cur.rs;
            R.V = V;
            R.Fin = sel3(a.F0, a.F1, a.F2, iin);
            R.Fout = sel3(a.F0, a.F1, a.F2, iout);
            R.Qpre_in = qin ? a.Qpre1 : a.Qpre0;
            R.Qrs_in = qin ? a.Qrs1 : a.Qrs0;
            R.TF_in = qin ? a.TF1 : a.TF0;
            R.Qpre_out = qout ? a.Qpre1 : a.Qpre0;
            R.Qrs_out = qout ? a.Qrs1 : a.Qrs0;
            R.TF_out = qout ? a.TF1 : a.TF0;
            R.qpack_out = slots + kSlotWords * iout;
            R.cap = dir == DIR_PUSH ? a.n : a.pull_cap;
            R.items_in = fused ? (uint64_t)m1 : items;
            R.mf = fused ? mf2 : mf;
            R.solo = dir == DIR_PUSH && a.stage &&
                     R.mf <= min((uint64_t)1 << a.tile_log2, (uint64_t)kStage);
            if (dir == DIR_PUSH) push_round<E, BLOCK>(a, R, s_pre, s_rs, sh, st_pre, st_rs, st_d);
            else pull_round<E, BLOCK>(a, R, sh, s_winc, s_wpos, st_pre, st_rs, st_d);
            // Round 1 also prepares the next query's visited bitmap (after the
            // round's own work, so the look-ahead loads have landed by then).
            if (r == 1) prep_visited(a, Vnext, qn < a.nq, nxt.s, gtid, gthreads);
            flush_round<E, BLOCK>(a, R, sh, st_pre, st_rs, st_d, slots + kSlotWords * iout);
            // After the last round only CTA 0 (which writes the result) needs
            // the counters.  While the barrier of round 1 waits, the last CTA
            // pulls the next query's seed row and its heads' row offsets into
            // L2 (prefetch only: nothing of that query is computed yet).
            const bool pf = r == 1 && qn < a.nq && blockIdx.x == gridDim.x - 1;
            const E pf_rs = nxt.rs;
            const uint64_t pf_d = min((uint64_t)(nxt.re - nxt.rs), (uint64_t)kPrefetchEdges);
            const auto prefetch_next = [&](unsigned t, unsigned nt) {
                if (!pf) return;
                for (uint64_t e = t; e < pf_d; e += nt) prefetch_l2(a.rp + a.ci[(uint64_t)pf_rs + e]);
            };
            // After a query's last round, the next query's fused prelude (it
            // reads only the graph and fills this CTA's shared tables) runs
            // between this CTA's arrival and its wait.
            const bool do_pre = R.last && qn < a.nq && nxt.k >= 2 && !all_pull && a.stage &&
                                (uint64_t)(nxt.re - nxt.rs) <= (uint64_t)kFuseDeg;
            const auto pre_next = [&]() {
                if (!do_pre) return;
                if (fused) {
                    prelude_clear<BLOCK>(s_nbr, s_npos, s_pslot, sh);
                    __syncthreads();
                }
                pre_m1 = fused_prelude<E, BLOCK>(a, nxt.s, nxt.rs, (uint32_t)(nxt.re - nxt.rs), s_nbr, s_npos,
                                                 s_pslot, s_pre, s_rs, sh);
            };
            if (!grid_barrier(&a.ctl->bar, &a.ctl->err, &sh.flag, bsense, slots + kSlotWords * iout, sh.slot,
                              (R.last && blockIdx.x != 0) ? 0 : 4, a.timeout_ns, prefetch_next, pre_next))
                return;
            pre_have = do_pre;
            const unsigned long long qp = sh.slot[0];
            const uint64_t nnew = sh.slot[1];
            const uint64_t scn = sh.slot[2];
            const uint64_t W = sizeof(E);
            const uint64_t items_out = R.last ? 0 : min((uint64_t)(qp >> a.ebits), R.cap);
            if (fused) {
                // rounds 1 and 2: q_1 (m1 vertices) was listed by every CTA
                if (!do_pre) prelude_clear<BLOCK>(s_nbr, s_npos, s_pslot, sh);
                if (b0) {
                    sh.q_bytes += 4ull * mf + (2ull * W + 4ull) + 4ull * m1;                   // round 1
                    sh.q_bytes += 4ull * mf2 + (2ull * W + 4ull) * m1 + 4ull * items_out;      // round 2
                    sh.q_te += mf2;
                    sh.q_count += m1 + nnew;
                    sh.q_rounds = 2u;
                }
                sum_mf += mf + mf2;
                visited += m1 + nnew;
                nf = nnew;
                items = qp >> a.ebits;
                mf = R.last ? 0 : sh.slot[3];
                prev = DIR_PUSH;
                if (b0 && a.per_hop) {
                    if (a.hop_stride > 1) a.per_hop[q * a.hop_stride + 1] = m1;
                    if (a.hop_stride > 2) a.per_hop[q * a.hop_stride + 2] = nnew;
                }
                r = 2;
                continue;
            }
            // Algorithmic bytes: push 4 m_f + (2W + 4) |F| + 4 |F_next| (edge
            // indices, row offsets and queue entries of the frontier, queue
            // entries of the next); pull n/8 (visited sweep) + n/8 (next
            // frontier) + 2W per unvisited vertex with in-edges + 4 per in-edge
            // scanned.
            if (b0) {
                if (dir == DIR_PUSH) {
                    sh.q_bytes += 4ull * mf + (2ull * W + 4ull) * (r == 1 ? 1ull : items) + 4ull * items_out;
                } else {
                    const uint64_t seen = visited + a.n_noin;
                    const uint64_t unvisited = a.n > seen ? a.n - seen : 0;
                    sh.q_bytes += 2ull * ((a.n + 7) / 8) + 2ull * W * unvisited + 4ull * scn;
                }
                sh.q_count += nnew;
                sh.q_rounds = r;
                if (dir == DIR_PULL && r <= 32) sh.q_pull |= 1u << (r - 1);
            }
            sum_mf += mf;
            visited += nnew;
            nf = nnew;
            items = qp >> a.ebits;
            mf = R.last ? 0 : sh.slot[3];
            prev = dir;
            if (b0 && a.per_hop && r < a.hop_stride) a.per_hop[q * a.hop_stride + r] = nnew;
        }
        if (b0) {
            const uint64_t now = globaltimer_ns();
            a.out[q] = sh.q_count;
            if (a.out_te) a.out_te[q] = sh.q_te;
            if (a.stats) {
                khop_query_stats st{t_prev, now, sh.q_te, sh.q_bytes, sh.q_rounds, sh.q_pull};
                a.stats[q] = st;
            }
            if (a.per_hop) {
                if (a.hop_stride) a.per_hop[q * a.hop_stride] = 1ull;
                for (uint64_t r = (uint64_t)sh.q_rounds + 1; r < a.hop_stride; ++r)
                    a.per_hop[q * a.hop_stride + r] = 0ull;
            }
            t_prev = now;
            if (qn > q + 1)   // answer the trivial queries up to qn
                skip_trivial(a, q + 1, true, t_prev, (QueryHead<E> *)nullptr);
        }
        q = qn;
        cur = nxt;
        par ^= 1u;
    }
}

// Dynamic shared memory of plain_kernel: push tile items, staging area and
// the fused round's hash set with its first-position table and slot list.
template <typename E>
size_t plain_smem_bytes(uint32_t tile_log2) {
    const size_t tcap = std::max<size_t>(size_t(1) << tile_log2, kFuseDeg) + 2;
    return (2 * tcap + 3 * (size_t)kStage) * sizeof(E) + 2 * (size_t)kHashSlots * sizeof(uint32_t) +
           (size_t)kFuseDeg * sizeof(uint16_t);
}

template <typename E, int BLOCK>
int launch_block(khop_graph *g, PlainArgs<E> &a, size_t smem, int grid_ctas, cudaStream_t st) {
    const void *fn = (const void *)plain_kernel<E, BLOCK>;
    int grid = 0;
    int rc = launch_shape(fn, BLOCK, smem, g->tune.blocks_per_sm, g->num_sms, &grid);
    if (rc != KHOP_OK) return rc;
    if (grid_ctas > 0 && grid_ctas < grid) grid = grid_ctas;
    cudaError_t e = cudaMemsetAsync(a.ctl, 0, offsetof(CtlBlock, err), st);   // keeps the sticky err
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BLOCK), args, smem, st);
    return cuda_status(e);
}

template <typename E>
int launch_typed(khop_graph *g, PlainState &ps, const uint32_t *seeds, const uint32_t *ks,
                 uint32_t k_all, uint64_t nq, uint64_t *out, uint64_t *out_te,
                 khop_query_stats *stats, uint64_t *per_hop, uint32_t hop_stride, int grid_ctas,
                 cudaStream_t st, bool keep_visited = false, int32_t *levels = nullptr,
                 bool take_test_switch = true) {
    PlainArgs<E> a;
    a.n = g->n;
    a.nnz = g->nnz;
    a.n_noin = g->n_noin;
    a.nw = g->nw;
    a.symmetric = g->symmetric ? 1 : 0;
    a.rp = (const E *)g->rp;
    a.ci = g->ci;
    a.cp = (const E *)g->cp;
    a.ri = g->ri;
    a.noin = g->noin;
    a.V0 = ps.V;
    a.V1 = ps.V2;
    a.F0 = ps.F[0];
    a.F1 = ps.F[1];
    a.F2 = ps.F[2];
    a.Qpre0 = (E *)ps.Qpre[0];
    a.Qpre1 = (E *)ps.Qpre[1];
    a.Qrs0 = (E *)ps.Qrs[0];
    a.Qrs1 = (E *)ps.Qrs[1];
    a.TF0 = ps.TF[0];
    a.TF1 = ps.TF[1];
    a.ctl = ps.ctl;
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
    a.keep_v = keep_visited || levels ? 1 : 0;
    a.levels = levels;
    a.alpha_fx = factor_fx16(g->tune.alpha);
    a.beta_fx = factor_fx16(g->tune.beta);
    uint32_t tl = 0;
    while ((1u << tl) < (uint32_t)g->tune.push_tile) ++tl;
    a.tile_log2 = tl;
    a.ebits = g->ebits;
    a.stage = g->nnz < (1ull << kStagePosShift) ? 1 : 0;
    a.pull_cap = g->tune.direction == KHOP_DIR_PULL
                     ? 0ull
                     : std::min<uint64_t>(g->n, (uint64_t)std::ceil((double)g->n / g->tune.beta) + 32);
    a.timeout_ns = g->timeout_ns;
    a.absent_at = 0;
    if (take_test_switch) {
        a.absent_at = g->absent_at;   // one launch only
        g->absent_at = 0;
    }
    const size_t smem = plain_smem_bytes<E>(tl);
    switch (g->tune.block_threads) {
        case 256: return launch_block<E, 256>(g, a, smem, grid_ctas, st);
        case 1024: return launch_block<E, 1024>(g, a, smem, grid_ctas, st);
        default: return launch_block<E, 512>(g, a, smem, grid_ctas, st);
    }
}

}  // namespace

int plain_launch(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint32_t k_all,
                 uint64_t nq, uint64_t *out, uint64_t *out_te, khop_query_stats *stats,
                 uint64_t *per_hop, uint32_t hop_stride, cudaStream_t st, bool keep_visited,
                 int32_t *levels) {
    if (g->ewidth == 4)
        return launch_typed<uint32_t>(g, g->plain, seeds, ks, k_all, nq, out, out_te, stats,
                                      per_hop, hop_stride, 0, st, keep_visited, levels);
    return launch_typed<unsigned long long>(g, g->plain, seeds, ks, k_all, nq, out, out_te,
                                            stats, per_hop, hop_stride, 0, st, keep_visited, levels);
}

int plain_launch_state(khop_graph *g, PlainState &ps, const uint32_t *seeds, const uint32_t *ks,
                       uint64_t nq, uint64_t *out, int grid_ctas, cudaStream_t st) {
    // (a server's launch: the graph's testing switch is left for the graph's own calls)
    if (g->ewidth == 4)
        return launch_typed<uint32_t>(g, ps, seeds, ks, 0, nq, out, nullptr, nullptr, nullptr, 0,
                                      grid_ctas, st, false, nullptr, false);
    return launch_typed<unsigned long long>(g, ps, seeds, ks, 0, nq, out, nullptr, nullptr,
                                            nullptr, 0, grid_ctas, st, false, nullptr, false);
}

}  // namespace khop

// ===========================================================================
// Allocation-free variant of the plain count (khop_count_static).
//
// Its traversal state lives in one file-scope device array of fixed size,
// so the entry point never allocates device memory.  Every GPU that loads
// the library holds the array until the process exits.  Host code reaches
// it only through the address cudaGetSymbolAddress returns for the current
// device (the array's name in host code is a host-side stand-in, not a
// device address).

namespace khop {
namespace {

constexpr uint64_t kStaticMaxN = 1ull << 20;      // vertices
constexpr uint64_t kStaticMaxNnz = 1ull << 26;    // edges
constexpr uint64_t kStaticNw = kStaticMaxN / 32;
constexpr uint64_t kStaticTF = kStaticMaxNnz / 256 + 2;   // push tiles of >= 256 edges
constexpr uint64_t kWordsPer256 = 64;
constexpr uint64_t round64(uint64_t x) { return (x + kWordsPer256 - 1) / kWordsPer256 * kWordsPer256; }
// layout in 32-bit words, every part 256-byte aligned
constexpr uint64_t kOffCtl = 0;
constexpr uint64_t kOffBits = round64(sizeof(CtlBlock) / 4);         // V0 V1 F0 F1 F2 noin
constexpr uint64_t kOffQ = kOffBits + 6 * round64(kStaticNw);        // Qpre0 Qpre1 Qrs0 Qrs1
constexpr uint64_t kOffTF = kOffQ + 4 * round64(kStaticMaxN);        // TF0 TF1
constexpr uint64_t kStaticWords = kOffTF + 2 * round64(kStaticTF);

static __device__ __align__(256) uint32_t g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint32_t *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once
// per device, with that device current).  The address is kept for the life
// of the process: it belongs to the device's primary context, so it does not
// survive cudaDeviceReset() or any other destruction of that context.
int static_scratch(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return KHOP_EINVAL;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_static_ptr[dev] = (uint32_t *)p;
    }
    *out = g_static_ptr[dev];
    return KHOP_OK;
}

// noin bitmap from a 32-bit CSC (or all zero without one).
__global__ void static_noin_kernel(const uint32_t *cp, uint64_t n, uint32_t nw, uint32_t *noin) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw; i += stride) {
        uint32_t w = 0;
        if (cp)
            for (int l = 0; l < 32; ++l) {
                const uint64_t v = (i << 5) + l;
                if (v < n && cp[v + 1] == cp[v]) w |= 1u << l;
            }
        noin[i] = w;
    }
}

}  // namespace
}  // namespace khop

extern "C" int khop_count_static(uint64_t n, const uint32_t *row_ptr, const uint32_t *col_idx,
                                 const uint32_t *col_ptr, const uint32_t *row_idx, uint64_t nnz,
                                 const uint32_t *seeds, uint64_t nseeds, uint32_t k,
                                 uint64_t *out_counts, void *stream) {
    using namespace khop;
    if (n == 0 || n > kStaticMaxN || nnz > kStaticMaxNnz) return KHOP_EINVAL;
    if (!row_ptr || (nnz && !col_idx) || (!col_ptr) != (!row_idx)) return KHOP_EINVAL;
    if (nseeds == 0) return KHOP_OK;
    if (!seeds || !out_counts) return KHOP_EINVAL;
    uint32_t *base = nullptr;
    int rc = static_scratch(&base);
    if (rc != KHOP_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);

    const uint32_t nw = (uint32_t)((n + 31) / 32);
    const bool has_csc = col_ptr != nullptr;
    PlainArgs<uint32_t> a;
    a.n = n;
    a.nnz = nnz;
    a.n_noin = 0;
    a.nw = nw;
    a.symmetric = (has_csc && col_ptr == row_ptr && row_idx == col_idx) ? 1 : 0;
    a.rp = row_ptr;
    a.ci = col_idx;
    a.cp = has_csc ? col_ptr : row_ptr;
    a.ri = has_csc ? row_idx : col_idx;
    uint32_t *bits = base + kOffBits;
    const uint64_t bw = round64(kStaticNw);
    a.V0 = bits;
    a.V1 = bits + bw;
    a.F0 = bits + 2 * bw;
    a.F1 = bits + 3 * bw;
    a.F2 = bits + 4 * bw;
    uint32_t *noin = bits + 5 * bw;
    a.noin = noin;
    const uint64_t qw = round64(kStaticMaxN);
    a.Qpre0 = base + kOffQ;
    a.Qpre1 = base + kOffQ + qw;
    a.Qrs0 = base + kOffQ + 2 * qw;
    a.Qrs1 = base + kOffQ + 3 * qw;
    a.TF0 = base + kOffTF;
    a.TF1 = base + kOffTF + round64(kStaticTF);
    a.ctl = (CtlBlock *)(base + kOffCtl);
    a.seeds = seeds;
    a.ks = nullptr;
    a.k_all = k;
    a.nq = nseeds;
    a.out = out_counts;
    a.out_te = nullptr;
    a.stats = nullptr;
    a.per_hop = nullptr;
    a.hop_stride = 0;
    a.direction = has_csc ? KHOP_DIR_AUTO : KHOP_DIR_PUSH;
    a.keep_v = 0;
    a.levels = nullptr;
    a.alpha_fx = factor_fx16(14.0f);
    a.beta_fx = factor_fx16(24.0f);
    a.tile_log2 = 11;   // 2048-edge push tiles
    uint32_t bl = 0;
    for (uint64_t x = n; x; x >>= 1) ++bl;
    a.ebits = 64 - bl;
    a.stage = 1;
    a.pull_cap = has_csc ? std::min<uint64_t>(n, (uint64_t)std::ceil((double)n / 24.0) + 32) : 0ull;
    a.timeout_ns = 2000000000ull;
    a.absent_at = 0;

    static_noin_kernel<<<nsm * 4, 256, 0, st>>>(col_ptr, n, nw, noin);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    constexpr int kBlk = 512;
    const size_t smem = plain_smem_bytes<uint32_t>(a.tile_log2);
    const void *fn = (const void *)plain_kernel<uint32_t, kBlk>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int grid = 0;
    rc = cooperative_grid(fn, kBlk, smem, 2, nsm, &grid);
    if (rc != KHOP_OK) return rc;
    e = cudaMemsetAsync(a.ctl, 0, sizeof(CtlBlock), st);   // counters, barrier and error word
    if (e != cudaSuccess) return cuda_status(e);
    // No error word survives the call, so a query the kernel does not finish
    // (a grid barrier that gave up) must not leave stale memory behind: every
    // count starts as UINT64_MAX and only a finished query overwrites it.
    e = cudaMemsetAsync(out_counts, 0xff, nseeds * sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlk), args, smem, st);
    return cuda_status(e);
}
