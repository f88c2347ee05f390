/*
 * CPU ORACLE for the k-hop neighbourhood count -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline use this file.  It is deliberately plain and slow, shares no code
 * with the CUDA library, and uses neither bitmaps, semirings nor a transposed
 * matrix.
 *
 * What it computes.  The paper benchmarks the "k-hop neighborhood count" for
 * k = 1, 2, 3 and 6 (Sec. III) on graphs stored as sparse adjacency matrices
 * whose traversals become sparse linear algebra (Sec. II).  For a seed s of a
 * directed graph with edges i -> j (A[i][j] = 1) the count is
 *
 *     | { u != s : dist(s, u) <= k } |
 *
 * where dist is the unweighted shortest-path length along edge direction.  The
 * masked (OR, AND) frontier iteration q <- (A^T q) AND NOT v, v <- v OR q
 * reaches exactly this set: after r rounds q holds the vertices at distance
 * exactly r and v those at distance <= r, so the count is |v| - 1.
 *
 * Algorithm: first-in first-out breadth-first search from s with a hop limit.
 *   dist[s] = 0, push s;
 *   pop u; if dist[u] == k do not expand; otherwise for every w in row u of
 *   the CSR with dist[w] unset: dist[w] = dist[u] + 1, count it, push w.
 * Duplicate edges and self-loops need no special case: a vertex is counted
 * only when its distance is first set, and s has distance 0 from the start.
 *
 * It also returns TE(s, k) = sum of outdeg(u) over all u with dist(s,u) < k:
 * the edges that a frontier-expanding (push) traversal examines, the
 * numerator of GTEPS.  per_hop[r] (optional) receives the number of vertices
 * at distance exactly r, r = 0..k.
 *
 * Portable C11 + pthreads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define UNSET (-1)

/* One query.  dist: int32[n], all UNSET on entry, restored to UNSET on exit.
 * queue: uint32[n] scratch.  Returns 0, or -1 for a seed out of range. */
int oracle_khop_one(uint64_t n, const uint64_t *row_ptr, const uint32_t *col_idx,
                    uint32_t s, uint32_t k, int32_t *dist, uint32_t *queue,
                    uint64_t *count, uint64_t *te, uint64_t *per_hop) {
    if ((uint64_t)s >= n) return -1;
    uint64_t head = 0, tail = 0, cnt = 0, edges = 0;
    if (per_hop) for (uint64_t r = 0; r <= k; ++r) per_hop[r] = 0;
    dist[s] = 0;
    queue[tail++] = s;
    if (per_hop) per_hop[0] = 1;
    while (head < tail) {
        uint32_t u = queue[head++];
        int32_t du = dist[u];
        if ((uint32_t)du >= k) continue;          /* at the hop limit: do not expand */
        edges += row_ptr[u + 1] - row_ptr[u];
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t w = col_idx[e];
            if (dist[w] == UNSET) {
                dist[w] = du + 1;
                cnt++;
                if (per_hop) per_hop[du + 1]++;
                queue[tail++] = w;
            }
        }
    }
    for (uint64_t i = 0; i < tail; ++i) dist[queue[i]] = UNSET;   /* restore */
    *count = cnt;
    if (te) *te = edges;
    return 0;
}

/* Distances from s for every vertex (UNSET = farther than k or unreachable). */
int oracle_khop_dist(uint64_t n, const uint64_t *row_ptr, const uint32_t *col_idx,
                     uint32_t s, uint32_t k, int32_t *dist_out) {
    if ((uint64_t)s >= n) return -1;
    uint32_t *queue = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!queue) return -2;
    for (uint64_t v = 0; v < n; ++v) dist_out[v] = UNSET;
    uint64_t head = 0, tail = 0;
    dist_out[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        uint32_t u = queue[head++];
        if ((uint32_t)dist_out[u] >= k) continue;
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t w = col_idx[e];
            if (dist_out[w] == UNSET) { dist_out[w] = dist_out[u] + 1; queue[tail++] = w; }
        }
    }
    free(queue);
    return 0;
}

/* Many independent queries, one query per thread at a time (the paper's
 * "each query runs in one thread", Sec. II).  counts[i] = UINT64_MAX for an
 * out-of-range seed.  te and per_hop may be NULL; per_hop is laid out as
 * per_hop[i * (hop_stride)] .. with hop_stride >= max k + 1. */
typedef struct {
    uint64_t n; const uint64_t *rp; const uint32_t *ci;
    const uint32_t *seeds; const uint32_t *ks; uint64_t nq;
    uint64_t *counts, *tes, *per_hop; uint64_t hop_stride;
    uint64_t next; int err;
} many_ctx;

static void *many_worker(void *arg) {
    many_ctx *c = (many_ctx *)arg;
    int32_t *dist = (int32_t *)malloc((c->n ? c->n : 1) * sizeof(int32_t));
    uint32_t *queue = (uint32_t *)malloc((c->n ? c->n : 1) * sizeof(uint32_t));
    if (!dist || !queue) {
        __atomic_store_n(&c->err, 1, __ATOMIC_RELAXED);
        free(dist); free(queue);
        return NULL;
    }
    for (uint64_t v = 0; v < c->n; ++v) dist[v] = UNSET;
    for (;;) {
        uint64_t i = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
        if (i >= c->nq) break;
        uint64_t cnt = 0, te = 0;
        uint64_t *ph = c->per_hop ? c->per_hop + i * c->hop_stride : NULL;
        if (ph && c->ks[i] + 1 > c->hop_stride) ph = NULL;
        if (oracle_khop_one(c->n, c->rp, c->ci, c->seeds[i], c->ks[i], dist, queue,
                            &cnt, &te, ph) != 0) {
            cnt = UINT64_MAX; te = UINT64_MAX;
        }
        c->counts[i] = cnt;
        if (c->tes) c->tes[i] = te;
    }
    free(dist); free(queue);
    return NULL;
}

int oracle_khop_many(uint64_t n, const uint64_t *row_ptr, const uint32_t *col_idx,
                     const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                     uint64_t *counts, uint64_t *tes, uint64_t *per_hop, uint64_t hop_stride,
                     int nthreads) {
    many_ctx c = {n, row_ptr, col_idx, seeds, ks, nq, counts, tes, per_hop, hop_stride, 0, 0};
    if (nthreads <= 0) {
        long cpus = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = cpus > 0 ? (int)cpus : 1;
    }
    if ((uint64_t)nthreads > nq) nthreads = nq ? (int)nq : 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, many_worker, &c) == 0) ++started;
    many_worker(&c);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return c.err ? -2 : 0;
}
