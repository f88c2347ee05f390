/*
 * Seeded synthetic inputs for the k-hop neighbourhood count: graphs, seed
 * vertices and request streams.  This module holds none of the counting
 * method; it only makes inputs.  Both the CPU oracle and the CUDA library are
 * fed from here, so both see identical graphs and seeds.
 *
 * Workload shapes follow the paper's benchmark (Sec. III): a Graph500-style
 * Kronecker/R-MAT graph and a Twitter-like power-law graph.
 *
 * Random numbers: a counter-based splitmix64 (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).  Draw i of stream
 * `key` is mix64(mix64(key) + (i + 1) * GAMMA), i.e. the i-th output of a
 * splitmix64 generator whose state starts at mix64(key).  Every draw is
 * addressed by its index, so results do not depend on the thread count.
 *
 * R-MAT: Chakrabarti, Zhan, Faloutsos, "R-MAT: A recursive model for graph
 * mining", SDM 2004: each edge picks one of four adjacency quadrants per level
 * with probabilities (A, B, C, D), most significant bit first.
 *
 * Chung-Lu: Chung and Lu, "Connected components in random graphs with given
 * expected degree sequences", 2002: an edge (u, v) is drawn with probability
 * proportional to w_out(u) * w_in(v).  Sampling uses Walker's alias method
 * (Walker 1977, "An efficient method for generating discrete random variables
 * with general distributions").
 *
 * Portable C11 + pthreads; no architecture-specific code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw i of the counter-based stream `key`. */
uint64_t khopgen_rand(uint64_t key, uint64_t i) {
    return mix64(mix64(key) + (i + 1) * GAMMA);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unif_from(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

double khopgen_unif(uint64_t key, uint64_t i) { return unif_from(khopgen_rand(key, i)); }

/* Fill out[j] = draw (start + j) of stream key, j < cnt. */
void khopgen_rand_fill(uint64_t key, uint64_t start, uint64_t cnt, uint64_t *out) {
    uint64_t base = mix64(key);
    for (uint64_t j = 0; j < cnt; ++j) out[j] = mix64(base + (start + j + 1) * GAMMA);
}

static int default_threads(int nt) {
    if (nt > 0) return nt;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

/* ------------------------------------------------------------------ */
/* Generic parallel-for over [0, total) in contiguous chunks.          */
typedef void (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void *ctx; uint64_t total, chunk; uint64_t next; } pfor_t;

static void *pfor_worker(void *arg) {
    pfor_t *p = (pfor_t *)arg;
    for (;;) {
        uint64_t lo = __atomic_fetch_add(&p->next, p->chunk, __ATOMIC_RELAXED);
        if (lo >= p->total) break;
        uint64_t hi = lo + p->chunk < p->total ? lo + p->chunk : p->total;
        p->fn(p->ctx, lo, hi);
    }
    return NULL;
}

static void pfor(range_fn fn, void *ctx, uint64_t total, uint64_t chunk, int nthreads) {
    if (total == 0) return;
    pfor_t p = {fn, ctx, total, chunk ? chunk : 1, 0};
    nthreads = default_threads(nthreads);
    pthread_t th[64];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, pfor_worker, &p) == 0) ++started;
    pfor_worker(&p);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* R-MAT edge list                                                    */
typedef struct {
    uint64_t key; int scale; double a, ab, abc;
    uint32_t *src, *dst;
} rmat_ctx;

static void rmat_range(void *vc, uint64_t lo, uint64_t hi) {
    rmat_ctx *c = (rmat_ctx *)vc;
    uint64_t base = mix64(c->key);
    for (uint64_t e = lo; e < hi; ++e) {
        uint32_t s = 0, d = 0;
        for (int l = 0; l < c->scale; ++l) {
            double u = unif_from(mix64(base + (e * (uint64_t)c->scale + (uint64_t)l + 1) * GAMMA));
            uint32_t sb, db;
            if (u < c->a) { sb = 0; db = 0; }
            else if (u < c->ab) { sb = 0; db = 1; }
            else if (u < c->abc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        c->src[e] = s;
        c->dst[e] = d;
    }
}

/* m = number of edges to draw (edge factor * 2^scale).  Edge e, level l uses
 * draw e*scale + l of stream `key`.  Vertex ids are NOT permuted here. */
int khopgen_rmat_edges(int scale, uint64_t m, double a, double b, double c,
                       uint64_t key, uint32_t *src, uint32_t *dst, int nthreads) {
    if (scale < 1 || scale > 32) return -1;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
    rmat_ctx ctx = {key, scale, a, a + b, a + b + c, src, dst};
    pfor(rmat_range, &ctx, m, 1u << 16, nthreads);
    return 0;
}

/* Seeded uniform random permutation of [0, n) by Fisher-Yates (Durstenfeld):
 * for i = n-1 .. 1 swap p[i] with p[j], j = draw(i) mod (i+1). */
void khopgen_permutation(uint64_t n, uint64_t key, uint32_t *perm) {
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    uint64_t base = mix64(key);
    for (uint64_t i = n; i-- > 1;) {
        uint64_t r = mix64(base + (i + 1) * GAMMA);
        uint64_t j = r % (i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

typedef struct { const uint32_t *perm; uint32_t *x; } relabel_ctx;
static void relabel_range(void *vc, uint64_t lo, uint64_t hi) {
    relabel_ctx *c = (relabel_ctx *)vc;
    for (uint64_t i = lo; i < hi; ++i) c->x[i] = c->perm[c->x[i]];
}
void khopgen_relabel(const uint32_t *perm, uint32_t *x, uint64_t m, int nthreads) {
    relabel_ctx ctx = {perm, x};
    pfor(relabel_range, &ctx, m, 1u << 16, nthreads);
}

/* ------------------------------------------------------------------ */
/* Edge list -> CSR with self-loop removal, optional symmetrisation    */
/* and duplicate collapse.  Rows come out sorted, so the result does    */
/* not depend on thread scheduling.                                     */
typedef struct {
    uint64_t n, m; const uint32_t *src, *dst; int sym;
    uint64_t *deg;      /* atomically incremented counts, then cursors */
    uint32_t *tmp;      /* scattered columns */
    uint64_t *off;      /* row offsets into tmp (n+1) */
    uint64_t *udeg;     /* unique degree per row */
    uint64_t *row_ptr;  /* output */
    uint32_t *col;      /* output */
} csr_ctx;

static void count_range(void *vc, uint64_t lo, uint64_t hi) {
    csr_ctx *c = (csr_ctx *)vc;
    for (uint64_t e = lo; e < hi; ++e) {
        uint32_t s = c->src[e], d = c->dst[e];
        if (s == d) continue;
        __atomic_fetch_add(&c->deg[s], 1, __ATOMIC_RELAXED);
        if (c->sym) __atomic_fetch_add(&c->deg[d], 1, __ATOMIC_RELAXED);
    }
}

static void scatter_range(void *vc, uint64_t lo, uint64_t hi) {
    csr_ctx *c = (csr_ctx *)vc;
    for (uint64_t e = lo; e < hi; ++e) {
        uint32_t s = c->src[e], d = c->dst[e];
        if (s == d) continue;
        uint64_t p = __atomic_fetch_add(&c->deg[s], 1, __ATOMIC_RELAXED);
        c->tmp[p] = d;
        if (c->sym) {
            uint64_t q = __atomic_fetch_add(&c->deg[d], 1, __ATOMIC_RELAXED);
            c->tmp[q] = s;
        }
    }
}

static int cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

static void sort_rows_range(void *vc, uint64_t lo, uint64_t hi) {
    csr_ctx *c = (csr_ctx *)vc;
    for (uint64_t r = lo; r < hi; ++r) {
        uint32_t *x = c->tmp + c->off[r];
        uint64_t d = c->off[r + 1] - c->off[r];
        if (d > 24) {
            qsort(x, d, sizeof(uint32_t), cmp_u32);
        } else {
            for (uint64_t i = 1; i < d; ++i) {
                uint32_t v = x[i]; uint64_t j = i;
                while (j > 0 && x[j - 1] > v) { x[j] = x[j - 1]; --j; }
                x[j] = v;
            }
        }
        uint64_t u = 0;
        for (uint64_t i = 0; i < d; ++i)
            if (i == 0 || x[i] != x[i - 1]) x[u++] = x[i];
        c->udeg[r] = u;
    }
}

static void copy_rows_range(void *vc, uint64_t lo, uint64_t hi) {
    csr_ctx *c = (csr_ctx *)vc;
    for (uint64_t r = lo; r < hi; ++r)
        memcpy(c->col + c->row_ptr[r], c->tmp + c->off[r], c->udeg[r] * sizeof(uint32_t));
}

/* Phase 1: returns the number of unique edges (after self-loop removal,
 * symmetrisation and dedup) and keeps the work arrays in *handle; phase 2
 * (khopgen_csr_finish) writes row_ptr[n+1] and col[nnz] and frees them. */
typedef struct { csr_ctx c; int nthreads; } csr_handle;

int64_t khopgen_csr_begin(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                          int symmetrize, int nthreads, void **handle) {
    csr_handle *h = (csr_handle *)calloc(1, sizeof(csr_handle));
    if (!h) return -1;
    h->nthreads = nthreads;
    csr_ctx *c = &h->c;
    c->n = n; c->m = m; c->src = src; c->dst = dst; c->sym = symmetrize ? 1 : 0;
    c->deg = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    c->off = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    c->udeg = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    if (!c->deg || !c->off || !c->udeg) goto fail;
    pfor(count_range, c, m, 1u << 16, nthreads);
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; ++i) { c->off[i] = acc; acc += c->deg[i]; c->deg[i] = c->off[i]; }
    c->off[n] = acc;
    c->tmp = (uint32_t *)malloc((acc ? acc : 1) * sizeof(uint32_t));
    if (!c->tmp) goto fail;
    pfor(scatter_range, c, m, 1u << 16, nthreads);
    pfor(sort_rows_range, c, n, 4096, nthreads);
    uint64_t tot = 0;
    for (uint64_t i = 0; i < n; ++i) tot += c->udeg[i];
    *handle = h;
    return (int64_t)tot;
fail:
    free(c->deg); free(c->off); free(c->udeg); free(c->tmp); free(h);
    return -1;
}

void khopgen_csr_finish(void *handle, uint64_t *row_ptr, uint32_t *col) {
    csr_handle *h = (csr_handle *)handle;
    csr_ctx *c = &h->c;
    uint64_t acc = 0;
    for (uint64_t i = 0; i < c->n; ++i) { row_ptr[i] = acc; acc += c->udeg[i]; }
    row_ptr[c->n] = acc;
    c->row_ptr = row_ptr; c->col = col;
    pfor(copy_rows_range, c, c->n, 4096, h->nthreads);
    free(c->deg); free(c->off); free(c->udeg); free(c->tmp); free(h);
}

/* ------------------------------------------------------------------ */
/* Seeds: uniform with replacement over {u : outdeg(u) > 0}.           */
/* Seed i = eligible[floor(u_i * n_eligible)], u_i = draw i of key.    */
int64_t khopgen_seeds(uint64_t n, const uint64_t *row_ptr, uint64_t count, uint64_t key,
                      uint32_t *out) {
    uint64_t ne = 0;
    for (uint64_t v = 0; v < n; ++v) ne += row_ptr[v + 1] > row_ptr[v];
    if (ne == 0) return 0;
    uint32_t *el = (uint32_t *)malloc(ne * sizeof(uint32_t));
    if (!el) return -1;
    uint64_t j = 0;
    for (uint64_t v = 0; v < n; ++v) if (row_ptr[v + 1] > row_ptr[v]) el[j++] = (uint32_t)v;
    uint64_t base = mix64(key);
    for (uint64_t i = 0; i < count; ++i) {
        double u = unif_from(mix64(base + (i + 1) * GAMMA));
        uint64_t idx = (uint64_t)(u * (double)ne);
        if (idx >= ne) idx = ne - 1;
        out[i] = el[idx];
    }
    free(el);
    return (int64_t)ne;
}

/* ------------------------------------------------------------------ */
/* Walker alias table over weights w[0..n): prob[i] in [0,1], alias[i]. */
int khopgen_alias_build(uint64_t n, const double *w, double *prob, uint32_t *alias) {
    double tot = 0;
    for (uint64_t i = 0; i < n; ++i) tot += w[i];
    if (!(tot > 0)) return -1;
    uint32_t *small = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *large = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!small || !large) { free(small); free(large); return -1; }
    uint64_t ns = 0, nl = 0;
    for (uint64_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / tot;
        alias[i] = (uint32_t)i;
        if (prob[i] < 1.0) small[ns++] = (uint32_t)i; else large[nl++] = (uint32_t)i;
    }
    while (ns && nl) {
        uint32_t s = small[--ns], l = large[nl - 1];
        alias[s] = l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) { --nl; small[ns++] = l; }
    }
    while (nl) prob[large[--nl]] = 1.0;
    while (ns) prob[small[--ns]] = 1.0;
    free(small); free(large);
    return 0;
}

typedef struct {
    uint64_t key_src, key_dst, start; uint64_t n_out, n_in;
    const double *ps, *pd; const uint32_t *as, *ad;
    uint32_t *src, *dst;
} cl_ctx;

static inline uint32_t alias_pick(uint64_t r, uint64_t n, const double *prob, const uint32_t *alias) {
    /* disjoint halves of the draw: the high 32 bits pick the column (n < 2^32),
       the low 32 bits decide column vs alias */
    const uint64_t col = ((r >> 32) * n) >> 32;
    const double u = (double)(r & 0xffffffffULL) * 0x1.0p-32;
    return u < prob[col] ? (uint32_t)col : alias[col];
}

static void cl_range(void *vc, uint64_t lo, uint64_t hi) {
    cl_ctx *c = (cl_ctx *)vc;
    uint64_t bs = mix64(c->key_src), bd = mix64(c->key_dst);
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t i = c->start + e;
        uint64_t rs = mix64(bs + (i + 1) * GAMMA), rd = mix64(bd + (i + 1) * GAMMA);
        c->src[e] = alias_pick(rs, c->n_out, c->ps, c->as);
        c->dst[e] = alias_pick(rd, c->n_in, c->pd, c->ad);
    }
}

/* Chung-Lu edge candidates start .. start+cnt: src ~ alias(out), dst ~ alias(in). */
void khopgen_chunglu_edges(uint64_t n, const double *prob_out, const uint32_t *alias_out,
                           const double *prob_in, const uint32_t *alias_in,
                           uint64_t key_src, uint64_t key_dst, uint64_t start, uint64_t cnt,
                           uint32_t *src, uint32_t *dst, int nthreads) {
    cl_ctx ctx = {key_src, key_dst, start, n, n, prob_out, prob_in, alias_out, alias_in, src, dst};
    pfor(cl_range, &ctx, cnt, 1u << 16, nthreads);
}

/* ------------------------------------------------------------------ */
/* Open-loop Poisson request stream: arrival t_i (seconds, rate lam),  */
/* hop count k_i from a categorical distribution, seed vertex uniform  */
/* over eligible ids given by the caller.                               */
void khopgen_poisson(uint64_t count, double lam, uint64_t key,
                     const double *k_cdf, const uint32_t *k_vals, int nk,
                     uint64_t n_eligible, const uint32_t *eligible,
                     double *t, uint32_t *ks, uint32_t *seeds) {
    uint64_t base = mix64(key);
    double now = 0.0;
    for (uint64_t i = 0; i < count; ++i) {
        double u0 = unif_from(mix64(base + (3 * i + 1) * GAMMA));
        double u1 = unif_from(mix64(base + (3 * i + 2) * GAMMA));
        double u2 = unif_from(mix64(base + (3 * i + 3) * GAMMA));
        now += -log1p(-u0) / lam;
        t[i] = now;
        int j = 0;
        while (j < nk - 1 && u1 >= k_cdf[j]) ++j;
        ks[i] = k_vals[j];
        uint64_t idx = (uint64_t)(u2 * (double)n_eligible);
        if (idx >= n_eligible) idx = n_eligible - 1;
        seeds[i] = eligible[idx];
    }
}

/* ------------------------------------------------------------------ */
/* Power-law weights: w(i) = w_min / (1 - u_i (1 - w_min / w_max)),     */
/* u_i = (i + 1/2) / n -- the quantiles of the density p(w) ~ w^-2 on   */
/* [w_min, w_max] -- with w_min found by bisection so that the weights  */
/* sum to `total`.  Returns w_min (or -1 if no w_min fits).             */
static double pl_sum(uint64_t n, double w_min, double w_max) {
    double s = 0, c = 0;   /* Kahan summation */
    const double r = 1.0 - w_min / w_max;
    for (uint64_t i = 0; i < n; ++i) {
        const double u = ((double)i + 0.5) / (double)n;
        const double y = w_min / (1.0 - u * r) - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    return s;
}

double khopgen_powerlaw_weights(uint64_t n, double w_max, double total, double *w) {
    double lo = 1e-9, hi = w_max;
    if (pl_sum(n, hi, w_max) < total || pl_sum(n, lo, w_max) > total) return -1.0;
    for (int it = 0; it < 100 && hi - lo > 1e-12 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (pl_sum(n, mid, w_max) < total) lo = mid; else hi = mid;
    }
    const double w_min = 0.5 * (lo + hi);
    const double r = 1.0 - w_min / w_max;
    for (uint64_t i = 0; i < n; ++i) w[i] = w_min / (1.0 - (((double)i + 0.5) / (double)n) * r);
    return w_min;
}

/* ------------------------------------------------------------------ */
/* Chung-Lu graph with an exact-prefix dedup.  Candidates i = 0..m-1   */
/* are drawn (src ~ alias_out, dst ~ alias_in); self-loops dropped.    */
/* Each distinct edge keeps its first occurrence i.  The output is the */
/* set of distinct edges whose first occurrence is below M*, where M*  */
/* is the smallest multiple of 2^20 for which that set reaches         */
/* `target` edges (so the result is `target` edges plus less than one  */
/* 2^20 block's new edges).  Rows come out sorted.                     */
typedef struct {
    uint64_t n, m;
    const double *po, *pi; const uint32_t *ao, *ai;
    uint64_t ks, kd;
    uint32_t *src, *dst;
    uint64_t *deg, *off;        /* counts / cursors, offsets [n+1] */
    uint64_t *pair;             /* (dst << 32 | first index) per row */
    uint64_t *udeg;             /* unique entries per row */
    uint64_t *hist;             /* [nthreads][nblk] first-occurrence block histogram */
    uint64_t nblk; int nthreads;
    uint64_t mstar;             /* cut: keep first occurrence < mstar */
    uint64_t *kdeg;             /* kept entries per row */
    uint64_t *row_ptr; uint32_t *col;
    uint64_t next_row;          /* dynamic row scheduling */
} cl_build;

static void clb_gen(void *vc, uint64_t lo, uint64_t hi) {
    cl_build *c = (cl_build *)vc;
    uint64_t bs = mix64(c->ks), bd = mix64(c->kd);
    for (uint64_t i = lo; i < hi; ++i) {
        c->src[i] = alias_pick(mix64(bs + (i + 1) * GAMMA), c->n, c->po, c->ao);
        c->dst[i] = alias_pick(mix64(bd + (i + 1) * GAMMA), c->n, c->pi, c->ai);
    }
}

static void clb_count(void *vc, uint64_t lo, uint64_t hi) {
    cl_build *c = (cl_build *)vc;
    for (uint64_t i = lo; i < hi; ++i)
        if (c->src[i] != c->dst[i]) __atomic_fetch_add(&c->deg[c->src[i]], 1, __ATOMIC_RELAXED);
}

static void clb_scatter(void *vc, uint64_t lo, uint64_t hi) {
    cl_build *c = (cl_build *)vc;
    for (uint64_t i = lo; i < hi; ++i) {
        const uint32_t s = c->src[i], d = c->dst[i];
        if (s == d) continue;
        const uint64_t p = __atomic_fetch_add(&c->deg[s], 1, __ATOMIC_RELAXED);
        c->pair[p] = ((uint64_t)d << 32) | (uint64_t)(uint32_t)i;
    }
}

static int cmp_u64(const void *x, const void *y) {
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* rows: sort pairs, keep the first occurrence of each dst, count per block */
typedef struct { cl_build *c; int tid; } clb_arg;
static void *clb_rows(void *va) {
    clb_arg *A = (clb_arg *)va;
    cl_build *c = A->c;
    uint64_t *h = c->hist + (uint64_t)A->tid * c->nblk;
    for (;;) {
        uint64_t lo = __atomic_fetch_add(&c->next_row, 1024, __ATOMIC_RELAXED);
        if (lo >= c->n) break;
        uint64_t hi = lo + 1024 < c->n ? lo + 1024 : c->n;
        for (uint64_t r = lo; r < hi; ++r) {
            uint64_t *x = c->pair + c->off[r];
            const uint64_t d = c->off[r + 1] - c->off[r];
            if (d > 1) qsort(x, d, sizeof(uint64_t), cmp_u64);
            uint64_t u = 0;
            for (uint64_t j = 0; j < d; ++j)
                if (u == 0 || (x[j] >> 32) != (x[u - 1] >> 32)) x[u++] = x[j];   /* min index first */
            c->udeg[r] = u;
            for (uint64_t j = 0; j < u; ++j) h[(x[j] & 0xffffffffULL) >> 20]++;
        }
    }
    return NULL;
}

static void clb_keep(void *vc, uint64_t lo, uint64_t hi) {
    cl_build *c = (cl_build *)vc;
    for (uint64_t r = lo; r < hi; ++r) {
        uint64_t *x = c->pair + c->off[r];
        uint64_t k = 0;
        for (uint64_t j = 0; j < c->udeg[r]; ++j)
            if ((x[j] & 0xffffffffULL) < c->mstar) x[k++] = x[j];
        c->kdeg[r] = k;
    }
}

static void clb_copy(void *vc, uint64_t lo, uint64_t hi) {
    cl_build *c = (cl_build *)vc;
    for (uint64_t r = lo; r < hi; ++r) {
        const uint64_t *x = c->pair + c->off[r];
        uint32_t *o = c->col + c->row_ptr[r];
        for (uint64_t j = 0; j < c->kdeg[r]; ++j) o[j] = (uint32_t)(x[j] >> 32);
    }
}

/* Returns the number of edges kept (>= target), or -1 (memory / m too
 * large for 32-bit indices), or -2 (m candidates give fewer than target
 * distinct edges: call again with a larger m).  *mstar_out = M*. */
int64_t khopgen_chunglu_begin(uint64_t n, const double *prob_out, const uint32_t *alias_out,
                              const double *prob_in, const uint32_t *alias_in,
                              uint64_t key_src, uint64_t key_dst, uint64_t m, uint64_t target,
                              int nthreads, uint64_t *mstar_out, void **handle) {
    if (m >= (1ULL << 32)) return -1;
    nthreads = default_threads(nthreads);
    cl_build *c = (cl_build *)calloc(1, sizeof(cl_build));
    if (!c) return -1;
    c->n = n; c->m = m; c->po = prob_out; c->pi = prob_in; c->ao = alias_out; c->ai = alias_in;
    c->ks = key_src; c->kd = key_dst; c->nthreads = nthreads;
    c->nblk = (m >> 20) + 1;
    c->src = (uint32_t *)malloc(m * sizeof(uint32_t));
    c->dst = (uint32_t *)malloc(m * sizeof(uint32_t));
    c->deg = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    c->off = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    c->udeg = (uint64_t *)malloc(n * sizeof(uint64_t));
    c->kdeg = (uint64_t *)malloc(n * sizeof(uint64_t));
    c->hist = (uint64_t *)calloc((uint64_t)nthreads * c->nblk, sizeof(uint64_t));
    if (!c->src || !c->dst || !c->deg || !c->off || !c->udeg || !c->kdeg || !c->hist) goto fail;
    pfor(clb_gen, c, m, 1u << 20, nthreads);
    pfor(clb_count, c, m, 1u << 20, nthreads);
    uint64_t acc = 0;
    for (uint64_t v = 0; v < n; ++v) { c->off[v] = acc; acc += c->deg[v]; c->deg[v] = c->off[v]; }
    c->off[n] = acc;
    c->pair = (uint64_t *)malloc((acc ? acc : 1) * sizeof(uint64_t));
    if (!c->pair) goto fail;
    pfor(clb_scatter, c, m, 1u << 20, nthreads);
    free(c->src); c->src = NULL;
    free(c->dst); c->dst = NULL;
    {
        pthread_t th[64];
        clb_arg args[64];
        int started = 0;
        for (int t = 0; t < nthreads && t < 64; ++t) {
            args[t].c = c; args[t].tid = t;
            if (t == 0) continue;
            if (pthread_create(&th[started], NULL, clb_rows, &args[t]) == 0) ++started;
            else args[t].tid = -1;
        }
        clb_rows(&args[0]);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    /* smallest block boundary reaching the target */
    uint64_t cum = 0, blk = 0;
    for (; blk < c->nblk; ++blk) {
        for (int t = 0; t < nthreads; ++t) cum += c->hist[(uint64_t)t * c->nblk + blk];
        if (cum >= target) break;
    }
    if (cum < target) {
        /* free everything; the caller retries with more candidates */
        free(c->deg); free(c->off); free(c->udeg); free(c->kdeg); free(c->hist); free(c->pair); free(c);
        return -2;
    }
    c->mstar = (blk + 1) << 20;
    pfor(clb_keep, c, n, 4096, nthreads);
    *mstar_out = c->mstar;
    *handle = c;
    return (int64_t)cum;
fail:
    free(c->src); free(c->dst); free(c->deg); free(c->off); free(c->udeg); free(c->kdeg);
    free(c->hist); free(c->pair); free(c);
    return -1;
}

void khopgen_chunglu_finish(void *handle, uint64_t *row_ptr, uint32_t *col) {
    cl_build *c = (cl_build *)handle;
    uint64_t acc = 0;
    for (uint64_t v = 0; v < c->n; ++v) { row_ptr[v] = acc; acc += c->kdeg[v]; }
    row_ptr[c->n] = acc;
    c->row_ptr = row_ptr; c->col = col;
    pfor(clb_copy, c, c->n, 4096, c->nthreads);
    free(c->deg); free(c->off); free(c->udeg); free(c->kdeg); free(c->hist); free(c->pair); free(c);
}

/* ------------------------------------------------------------------ */
/* Checksum of a byte array, for the on-disk graph cache: the sum over  */
/* 8-byte words w_i (the tail zero-padded) of mix64(w_i ^ mix64(i + 1)), */
/* mod 2^64, finalised with the byte count.  Order-sensitive through the */
/* word index, independent of the thread count (the sum commutes).      */
typedef struct { const unsigned char *p; uint64_t nbytes; uint64_t *part; uint64_t chunk; } ck_ctx;

static void ck_range(void *vc, uint64_t lo, uint64_t hi) {
    ck_ctx *c = (ck_ctx *)vc;
    uint64_t acc = 0;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t w = 0;
        uint64_t off = i * 8;
        uint64_t take = c->nbytes - off < 8 ? c->nbytes - off : 8;
        memcpy(&w, c->p + off, take);
        acc += mix64(w ^ mix64(i + 1));
    }
    c->part[lo / c->chunk] = acc;
}

uint64_t khopgen_checksum(const void *p, uint64_t nbytes, int nthreads) {
    const uint64_t words = (nbytes + 7) / 8;
    const uint64_t chunk = 1ull << 20;
    const uint64_t nparts = (words + chunk - 1) / chunk;
    uint64_t *part = (uint64_t *)calloc(nparts ? nparts : 1, sizeof(uint64_t));
    if (!part) return 0;
    ck_ctx c = {(const unsigned char *)p, nbytes, part, chunk};
    pfor(ck_range, &c, words, chunk, nthreads);
    uint64_t h = 0;
    for (uint64_t i = 0; i < nparts; ++i) h += part[i];
    free(part);
    return mix64(h ^ nbytes);
}
