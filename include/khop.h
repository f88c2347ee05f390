/*
 * khop.h -- C ABI of libkhop, a GB300 (sm_103a) library for the k-hop
 * neighbourhood count.
 *
 * The operation.  RedisGraph (Cailliau et al., "RedisGraph GraphBLAS Enabled
 * Graph Database", Sec. II) keeps a graph as a sparse Boolean adjacency matrix
 * A (A[i][j] = 1 for an edge i -> j) and runs traversals as sparse linear
 * algebra; its benchmark query (Sec. III) is the k-hop neighbourhood count,
 * k = 1, 2, 3 and 6.  For a seed s this library returns
 *
 *     count(s, k) = | { u != s : u is reachable from s in 1..k hops } |
 *
 * computed GraphBLAS-style: q0 = v0 = {s}; for r = 1..k
 *     q_r = (A^T q_{r-1}) AND NOT v_{r-1}      over the (OR, AND) semiring
 *     v_r = v_{r-1} OR q_r
 * and count = popcount(v_k) - 1.  All arithmetic is integer: results are exact.
 *
 * Conventions for every call:
 *  - Each call returns a khop_status; nothing aborts the process or traps the
 *    GPU.  khop_strerror() gives a message.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that take device buffers are asynchronous and ordered on
 *    that stream; the caller synchronises.
 *  - A graph's traversal state is shared by the calls made on it: calls on one
 *    graph run one after another (the library orders calls made on different
 *    streams with events).  Different graphs are independent.
 *  - Device-side failures (a seed >= n, a device wait that ran out) are
 *    recorded in the graph's sticky error word, read by khop_get_error().
 */
#ifndef KHOP_H
#define KHOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
enum khop_status {
    KHOP_OK = 0,
    KHOP_EINVAL = 1,      /* bad argument (NULL, size, flag, malformed CSR)   */
    KHOP_ENOMEM = 2,      /* device or host allocation failed                 */
    KHOP_ECUDA = 3,       /* a CUDA runtime call failed                        */
    KHOP_EBUSY = 4,       /* admission refused: no memory or slot right now    */
    KHOP_ETIMEDOUT = 5,   /* a bounded device or host wait ran out             */
    KHOP_ESHUTDOWN = 6,   /* the server is shutting down                       */
    KHOP_EDEVICE = 7      /* a device-side error was recorded (khop_get_error) */
};

/* Sticky device error bits reported by khop_get_error(). */
enum khop_device_error {
    KHOP_DEVERR_TIMEOUT = 1,   /* a grid barrier or device wait gave up        */
    KHOP_DEVERR_SEED = 2,      /* a seed was >= n (its count is UINT64_MAX)   */
    KHOP_DEVERR_CAPACITY = 4   /* an internal capacity check failed           */
};

const char *khop_strerror(int status);
/* Library version: major * 10000 + minor * 100 + patch. */
int khop_version(void);

/* ---- graphs ------------------------------------------------------------ */
typedef struct khop_graph khop_graph;

enum khop_graph_flags {
    KHOP_HOST_PTRS = 0,     /* row_ptr / col_idx are host pointers             */
    KHOP_DEVICE_PTRS = 1,   /* row_ptr / col_idx are device pointers           */
    KHOP_SYMMETRIC = 2,     /* caller asserts A = A^T; the CSC is the CSR       */
    KHOP_VALIDATE = 4,      /* check the CSR (monotone row_ptr, row_ptr[n] =
                               nnz, col_idx < n) before use; EINVAL if not      */
    KHOP_WIDE_OFFSETS = 8,  /* keep 64-bit edge offsets on the device even when
                               nnz < 2^32 (otherwise they are stored 32-bit)    */
    KHOP_REVERSE = 16,      /* count in-neighbourhoods: q_r = A q_{r-1}, the
                               frontier expands along edges backwards (the graph
                               is stored transposed)                             */
    KHOP_UNDIRECTED = 32    /* count along edges in either direction:
                               q_r = (A OR A^T) q_{r-1}; the graph is stored as
                               the union of each vertex's out- and in-list
                               (2 nnz entries).  Overrides KHOP_REVERSE.         */
};

/*
 * Create a graph from CSR: row u lists the heads w of the edges u -> w (the
 * rows of the adjacency matrix A).  The transpose A^T (CSC, in-edges) is
 * derived on the device.  By default a query counts the out-neighbourhood
 * (Sec. III: q_r = A^T q_{r-1}); KHOP_REVERSE and KHOP_UNDIRECTED select the
 * in-neighbourhood and the either-direction neighbourhood, for every later
 * count, batch and server request on the graph.
 *   n              vertices, 1 <= n < 2^32 (col_idx is 32-bit)
 *   row_ptr        n+1 offsets, each row_ptr_bytes wide (4 or 8)
 *   col_idx        nnz uint32 column indices, each < n
 *   nnz            row_ptr[n]; bitlen(n) + bitlen(nnz) must be <= 64 (with
 *                  KHOP_UNDIRECTED: bitlen(n) + bitlen(2 nnz) <= 64)
 *   flags          khop_graph_flags
 *   stream         stream for the upload and the derivation
 *   out            receives the graph handle
 * Ownership: the inputs are copied and the call synchronises `stream` before
 * it returns, so the caller may free them when it returns.  The graph owns its device copies and its
 * traversal state.  Duplicate edges and self-loops are allowed and do not
 * change any count.
 * Errors: EINVAL (n, nnz, width, flags, NULL, or a failed KHOP_VALIDATE),
 * ENOMEM, ECUDA.
 */
int khop_graph_create(uint64_t n, const void *row_ptr, int row_ptr_bytes,
                      const uint32_t *col_idx, uint64_t nnz, uint32_t flags,
                      void *stream, khop_graph **out);

/* Free the graph and everything it owns (synchronises the device first). */
int khop_graph_destroy(khop_graph *g);

/* n and nnz of the graph (either pointer may be NULL). */
int khop_graph_info(const khop_graph *g, uint64_t *n, uint64_t *nnz);

/* Device memory held by the graph, in bytes (CSR, CSC and state pools). */
int khop_graph_device_bytes(const khop_graph *g, uint64_t *bytes);

/* ---- traversal tuning -------------------------------------------------- */
enum khop_direction {
    KHOP_DIR_AUTO = 0,   /* Beamer direction switch (push <-> pull)          */
    KHOP_DIR_PUSH = 1,   /* every round expands the frontier (SpMSpV)        */
    KHOP_DIR_PULL = 2    /* every round scans unvisited vertices (masked SpMV) */
};

/*
 * Tunables of a graph.  The direction switch follows Beamer, Asanovic and
 * Patterson, "Direction-optimizing breadth-first search" (SC 2012): switch
 * push -> pull when m_f > m_u / alpha and pull -> push when n_f < n / beta,
 * where n_f is the frontier size, m_f the out-edges of the frontier and m_u
 * the out-edges of unvisited vertices.  Fields set to 0 keep the current
 * value.  Changing the tuning never changes a count.
 */
typedef struct {
    int32_t direction;        /* khop_direction                                   */
    float alpha;              /* push -> pull threshold (> 0)                     */
    float beta;               /* pull -> push threshold (> 0)                     */
    int32_t block_threads;    /* threads per CTA of the traversal kernels: 256, 512 or 1024 */
    int32_t blocks_per_sm;    /* CTAs per SM (capped by occupancy)                */
    int32_t push_tile;        /* edges per push tile: power of two, 256 .. 8192   */
    float batch_alpha;        /* alpha for the 64-lane batched traversal          */
    float batch_beta;         /* beta for the 64-lane batched traversal           */
    int32_t batch_push_tile;  /* edges per push tile of the batched traversal: power of two, 256 .. 8192 */
} khop_tuning;

int khop_graph_get_tuning(const khop_graph *g, khop_tuning *t);
int khop_graph_set_tuning(khop_graph *g, const khop_tuning *t);

/*
 * Pick tuning values for this graph by timing candidate settings -- grid
 * shape, push tile, alpha and beta of the plain path, then alpha, beta and
 * push tile of the batched path -- on `nq` queries (device array `seeds`; per-seed hops in
 * the device array `ks`, or, if ks is NULL, `k` for every seed), keeping the
 * fastest of each, and apply them.  Synchronises `stream`.  Never changes a
 * count.
 */
int khop_autotune(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nq,
                  uint32_t k, void *stream, khop_tuning *chosen);

/* ---- counting ---------------------------------------------------------- */
/*
 * k-hop counts for nseeds seeds with the same k, on the plain single-query
 * path: the queries run one after another, each over the whole GPU
 * (direction-optimizing push/pull), inside one persistent launch.
 *   seeds        device uint32[nseeds]
 *   k            hops; k = 0 gives 0; large k is fine (stops when the
 *                frontier empties)
 *   out_counts   device uint64[nseeds]; a seed >= n gives UINT64_MAX and sets
 *                KHOP_DEVERR_SEED
 * Errors: EINVAL, ECUDA.  Asynchronous on `stream`.
 */
int khop_count(khop_graph *g, const uint32_t *seeds, uint64_t nseeds, uint32_t k,
               uint64_t *out_counts, void *stream);

enum khop_mode {
    KHOP_MODE_AUTO = 0,       /* batched for nseeds >= 2, else plain              */
    KHOP_MODE_PLAIN = 1,      /* one query at a time                              */
    KHOP_MODE_BATCHED64 = 2,  /* up to 64 queries share one bit-sliced traversal  */
    KHOP_MODE_BATCHED128 = 3, /* up to 128 queries share one traversal (two lane
                                 words per vertex)                              */
    KHOP_MODE_BATCHED256 = 4  /* up to 256 queries share one traversal (four lane
                                 words per vertex)                              */
};

/*
 * Per-seed k (ks[i] for seeds[i]).  In KHOP_MODE_BATCHED64 the queries are
 * grouped by k and packed 64 per uint64 lane word (KHOP_MODE_BATCHED128: 128
 * per pair of words; KHOP_MODE_BATCHED256: 256 per four words); every lane's result equals the same query run alone.  seeds, ks, out_counts: device arrays of nseeds.
 * After a first call with the same mode on g (which allocates the batch
 * state), khop_count, khop_count_ex and khop_count_mixed issue only stream
 * work, so they may be captured into a CUDA graph and replayed; the graph
 * then owns the ordering of its launches.
 */
int khop_count_mixed(khop_graph *g, const uint32_t *seeds, const uint32_t *ks,
                     uint64_t nseeds, uint64_t *out_counts, int mode, void *stream);

/*
 * Hop levels of one query's BFS (Sec. III's rounds as the (MIN, +) semiring)
 * and, optionally, BFS parents over the (MIN, SECOND) semiring.
 *   out_levels   device int32[n]: level(v) = hop distance from `seed` if it
 *                is <= k (0 for the seed), else -1
 *   out_parents  device uint32[n] or NULL: parent(v) = the smallest
 *                in-neighbour u of v with level(u) = level(v) - 1 for a
 *                reached v != seed; parent(seed) = seed; UINT32_MAX for
 *                unreached vertices.  Unique, so any correct BFS gives it.
 * On a KHOP_REVERSE / KHOP_UNDIRECTED graph "in-neighbour" follows the
 * traversal direction.  Asynchronous on `stream`, ordered with the graph's
 * other calls.  Errors: EINVAL (NULL graph or out_levels, seed >= n), ECUDA.
 */
int khop_levels(khop_graph *g, uint32_t seed, uint32_t k, int32_t *out_levels,
                uint32_t *out_parents, void *stream);

/*
 * One masked matrix-vector product over a semiring, the building block the
 * paper's Sec. II runs every traversal with (the k-hop count is the (OR, AND)
 * case iterated, masked by the complement of the visited set):
 *     y[v] = (+)_{u : A[u][v] = 1} x[u] (x) 1     for the vertices v the mask selects,
 *     y[v] = the (+)-identity                       for the others,
 * i.e. y = A^T x over in-edges (on a KHOP_REVERSE / KHOP_UNDIRECTED graph the
 * in-edges of the stored direction, as for every count).
 *   semiring   KHOP_SR_OR_AND:     y[v] = 1 if some in-neighbour u has x[u] != 0, else 0
 *              KHOP_SR_PLUS_TIMES: y[v] = sum of x[u] over the in-edges, mod 2^64
 *                                  (iterated from e_s: the number of walks of each length)
 *              KHOP_SR_MIN_SECOND: y[v] = min of x[u] over the in-edges, UINT64_MAX if
 *                                  none (x[u] = u on a frontier: BFS parents)
 *              KHOP_SR_MAX_SECOND: y[v] = max of x[u] over the in-edges, 0 if none
 *   x          device uint64[n]; the (+)-identity (0; UINT64_MAX for MIN) means "no entry"
 *   mask       device uint32 bitmap [ceil(n/32)] (bit v of word v/32) or NULL = all
 *              vertices; mask_complement != 0 selects the vertices whose bit is clear
 *   y          device uint64[n], written whole; may not alias x
 * Sums run over the stored in-edges: an edge given twice to khop_graph_create
 * adds twice.  Asynchronous on `stream`, ordered with the graph's other calls.
 * Errors: EINVAL (NULL graph / x / y, unknown semiring), ECUDA.
 */
enum khop_semiring {
    KHOP_SR_OR_AND = 0,
    KHOP_SR_PLUS_TIMES = 1,
    KHOP_SR_MIN_SECOND = 2,
    KHOP_SR_MAX_SECOND = 3
};
int khop_mxv(khop_graph *g, int semiring, const uint64_t *x, const uint32_t *mask, int mask_complement,
             uint64_t *y, void *stream);

/* In-edges examined by the last khop_mxv call on g (read it before the next
 * call on g; synchronises the device). */
int khop_mxv_stats(khop_graph *g, uint64_t *scanned);

/*
 * The k-hop neighbourhood itself -- the visited set v_k of Sec. III, the seed
 * included -- rather than its size, for one query on the plain path.
 *   khop_neighbourhood: bit v of out_bits (ceil(n/32) uint32 words, device
 *     memory, written whole) is set iff v is within k hops of `seed`;
 *     out_count (device uint64, may be NULL) receives the count
 *     (popcount - 1), as khop_count would.
 *   khop_neighbourhood_list: the same set as vertex ids in ascending order:
 *     the first min(size, capacity) ids go to out_ids (device uint32; may be
 *     NULL when capacity is 0) and the set's size to *out_size (device
 *     uint64), so a call with capacity 0 sizes the buffer for a second call.
 * Asynchronous on `stream` like khop_count; ordered with the graph's other
 * calls.  Errors: EINVAL (NULL graph or output, seed >= n), ECUDA.
 */
int khop_neighbourhood(khop_graph *g, uint32_t seed, uint32_t k, uint32_t *out_bits,
                       uint64_t *out_count, void *stream);
int khop_neighbourhood_list(khop_graph *g, uint32_t seed, uint32_t k, uint32_t *out_ids,
                            uint64_t capacity, uint64_t *out_size, void *stream);

/*
 * Counters of the last batched launch on g (either lane width): batches run, algorithmic HBM bytes (the method's compulsory traffic: lane
 * words of the vertices and frontier items touched, edge indices read,
 * harvest sweeps), rounds and pull rounds.  Synchronises the device.  Any
 * pointer may be NULL.
 */
int khop_batch_stats(khop_graph *g, uint64_t *batches, uint64_t *bytes, uint64_t *rounds,
                     uint64_t *pull_rounds);

/* Per-query record of the plain path (device memory, filled by khop_count_ex). */
typedef struct {
    uint64_t t_start_ns;   /* %globaltimer when the query's first round began  */
    uint64_t t_end_ns;     /* %globaltimer when its count was final           */
    uint64_t te;           /* TE(s,k): sum of out-degrees of vertices at distance < k */
    uint64_t bytes;        /* algorithmic HBM bytes of the rounds it ran       */
    uint32_t rounds;       /* rounds run (<= k; fewer if the frontier emptied) */
    uint32_t pull_mask;    /* bit r-1 set if round r ran as pull (r <= 32)    */
} khop_query_stats;

/*
 * khop_count with per-seed k and optional outputs of the plain path:
 *   out_te      device uint64[nseeds] or NULL: TE(s, k)
 *   out_stats   device khop_query_stats[nseeds] or NULL
 *   per_hop     device uint64[nseeds * hop_stride] or NULL: per_hop[i*stride + r]
 *               = vertices at distance exactly r (r = 0..min(k, stride-1))
 */
int khop_count_ex(khop_graph *g, const uint32_t *seeds, const uint32_t *ks, uint64_t nseeds,
                  uint64_t *out_counts, uint64_t *out_te, khop_query_stats *out_stats,
                  uint64_t *per_hop, uint32_t hop_stride, void *stream);

/*
 * khop_count without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * whose device memory is owned by another allocator (for example a
 * framework's caching pool that has reserved the GPU), and latency-critical
 * callers that cannot afford the implicit device synchronisation of an
 * allocation.  Such callers cannot create a khop_graph either, so they pass
 * the graph itself as device arrays.
 *   n            vertices, 1 <= n <= 2^20 (1,048,576)
 *   row_ptr      device uint32[n+1]: CSR row offsets (out-edges)
 *   col_idx      device uint32[nnz]: CSR heads
 *   col_ptr      device uint32[n+1] or NULL: CSC column offsets (in-edges)
 *   row_idx      device uint32[nnz] or NULL: CSC tails (NULL exactly when
 *                col_ptr is); with a CSC the traversal switches between push
 *                and pull, without one it only pushes.  Passing the CSR
 *                arrays again declares the graph symmetric.
 *   nnz          edges, <= 2^26 (67,108,864)
 *   seeds, nseeds, k, out_counts, stream: as for khop_count
 * The traversal state lives in one fixed device array of about 20 MB that
 * every GPU which loads this library holds until the process exits.  The
 * first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  All
 * calls share the array and the next call overwrites it, so calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race: order them on one stream.  Each call resets the state it needs.
 * The looked-up address belongs to the device's primary context: after
 * cudaDeviceReset() (or any other destruction of that context) in this
 * process, the entry point must not be called again on that device.
 * Errors: EINVAL for sizes beyond the limits or bad pointers, ECUDA.  No
 * sticky error word is kept: out_counts is first filled with UINT64_MAX and
 * a query overwrites its entry only when its count is final, so UINT64_MAX
 * marks a seed >= n or a query whose traversal did not finish (a device wait
 * that ran out).
 */
int khop_count_static(uint64_t n, const uint32_t *row_ptr, const uint32_t *col_idx,
                      const uint32_t *col_ptr, const uint32_t *row_idx, uint64_t nnz,
                      const uint32_t *seeds, uint64_t nseeds, uint32_t k,
                      uint64_t *out_counts, void *stream);

/*
 * Read and clear the graph's sticky device error bits (synchronises the
 * device).  After KHOP_DEVERR_TIMEOUT the launch that recorded it stopped
 * early: the outputs of its unfinished queries are undefined.  The graph
 * stays usable -- the next call starts from reset traversal state.
 */
int khop_get_error(khop_graph *g, uint32_t *device_error_bits);

/*
 * Bound of every device-side wait of the graph's traversals (the grid
 * barriers between rounds), in nanoseconds of %globaltimer; 0 restores the
 * default of 2 s; at most 60 s.  A wait that runs out records
 * KHOP_DEVERR_TIMEOUT and the launch leaves early instead of hanging.  The
 * limit must exceed the longest legitimate wait: one round of a traversal,
 * or, on the plain path, a run of up to 8192 one-CTA 1-hop queries that the
 * other CTAs wait out at one barrier.  Errors: EINVAL.
 */
int khop_graph_set_wait_limit(khop_graph *g, uint64_t timeout_ns);

/*
 * For testing failure detection without faulting the GPU: in the next
 * traversal launch on g (plain or batched, then the switch clears itself),
 * the grid's last CTA does not arrive at its barrier_index-th grid barrier
 * (1 = the first).  The other CTAs' bounded wait runs out, exactly as if that
 * CTA had been lost: KHOP_DEVERR_TIMEOUT is recorded and the launch returns;
 * the absent CTA sleeps until it sees the timeout (at most twice the wait
 * limit plus 1 ms) and leaves too.  0 switches it off.  Errors: EINVAL.
 */
int khop_graph_test_absent_cta(khop_graph *g, uint32_t barrier_index);

/* ---- serving ----------------------------------------------------------- */
/*
 * A request server: k-hop queries of mixed k arrive one by one on resident
 * graphs.  Heavy requests (k >= 3) are continuously batched at round
 * granularity: a rolling slot holds a 64-lane bit-sliced traversal on the
 * device and runs it one round per step (one launch); a step advances every
 * lane in use by one hop, whatever its depth.  Between steps a worker thread
 * posts the result of every lane the step retired -- its k-th round ran, or
 * its frontier came out empty, so its count is final -- and admits waiting
 * requests into the free lanes, each with its own round counter: a request
 * that arrives while a traversal runs joins it at the next round boundary.
 * Heavy requests of similar depth share a slot (one class for k = 3, one
 * for k >= 4), so a slot's lanes mostly retire together.  While at most
 * plain_heavy heavy requests wait, they take the single-query path instead.
 * Light requests (k <= 2) take a few microseconds each on the single-query
 * path, so plain slots answer them in arrival order, several per launch.
 * Slots (their device state) are admitted by free device memory and the
 * budget; the launches of different slots run side by side on the device.
 * This is the GPU counterpart of the paper's thread pool serving many
 * concurrent queries at low latency (Sec. II).
 */
typedef struct khop_server khop_server;

typedef struct {
    uint64_t mem_budget_bytes;   /* max device bytes for slot state (0 = no cap
                                    beyond free memory minus a 1 GiB margin)   */
    uint32_t max_batches;        /* max rolling 64-lane slots per graph (0 = 3;
                                    at most 3).  Slots hold one depth class:
                                    k = 3, or k >= 4; with 1 the single slot
                                    takes both                                  */
    int64_t wait_timeout_us;     /* bound for the worker's wait for a step
                                    (0 = 2 s; negative: EINVAL)                 */
    uint32_t max_pending;        /* max queued requests before EBUSY (0 = 1<<20) */
    uint32_t admit_rounds;       /* a rolling traversal admits new lanes while its
                                    lanes have run at most this many rounds
                                    (0 = 1; UINT32_MAX = at every step)          */
    int32_t plain_heavy;         /* heavy requests take the single-query path
                                    while at most this many wait (0 = 2;
                                    negative = never)                            */
} khop_server_opts;

typedef struct {
    uint64_t ticket;        /* as returned by khop_submit                      */
    uint64_t count;         /* the k-hop count (UINT64_MAX on error)           */
    int32_t status;         /* khop_status of this request                     */
    uint32_t k;             /* hops requested                                  */
    uint64_t t_submit_ns;   /* host CLOCK_MONOTONIC at submit                  */
    uint64_t t_done_ns;     /* host CLOCK_MONOTONIC when the result was posted */
} khop_result;

/* Create a server (starts its worker thread).  opts may be NULL. */
int khop_server_create(const khop_server_opts *opts, khop_server **out);

/*
 * Queue one request: count(seed, k) on graph g (g must outlive the server's
 * use of it).  Thread-safe.  Errors: EINVAL (seed >= n), EBUSY (queue full),
 * ESHUTDOWN.
 */
int khop_submit(khop_server *s, khop_graph *g, uint32_t seed, uint32_t k, uint64_t *ticket);

/*
 * Queue `count` requests at once (host arrays seeds[i], ks[i]); tickets[i]
 * receives each ticket.  All or nothing: EINVAL if any seed >= n, EBUSY if
 * the queue cannot take them all.  Thread-safe.
 */
int khop_submit_many(khop_server *s, khop_graph *g, const uint32_t *seeds, const uint32_t *ks,
                     uint32_t count, uint64_t *tickets);

/*
 * Take up to `max` finished results, waiting up to timeout_us (0 = do not
 * wait, < 0 = wait until at least one is available or the server stops).
 * *nout receives the number written.  Thread-safe.
 */
int khop_poll(khop_server *s, khop_result *out, uint32_t max, uint32_t *nout, int64_t timeout_us);

/* Server counters (any pointer may be NULL); batches_allocated = rolling slots allocated. */
int khop_server_stats(khop_server *s, uint64_t *submitted, uint64_t *completed,
                      uint64_t *steps, uint64_t *batches_allocated);

typedef struct {
    uint64_t submitted;        /* requests accepted by khop_submit / khop_submit_many  */
    uint64_t completed;        /* results posted (any status)                          */
    uint64_t steps;            /* step launches (one round of one slot each)           */
    uint64_t slots_allocated;  /* slots whose device state was admitted               */
    uint64_t joined_running;   /* requests admitted into a slot whose traversal was
                                  already running (continuous batching)               */
    uint64_t retired_early;    /* lanes retired before their k-th round: the frontier
                                  came out empty                                      */
    uint64_t timed_out;        /* requests completed with KHOP_ETIMEDOUT              */
    uint64_t max_lanes_busy;   /* most lanes in use at once, over all slots           */
    uint64_t gpu_step_ns;      /* device time of the steps (sum of their durations)   */
    uint64_t pull_steps;       /* steps whose round ran as a pull                    */
    uint64_t clean_steps;      /* steps asked to sweep retired lanes' marks away      */
    uint64_t lane_steps;       /* sum over steps of the lanes they advanced           */
    uint64_t plain_launches;   /* launches of the single-query path (light requests)  */
} khop_server_counters;

/* All server counters at once.  Errors: EINVAL. */
int khop_server_counters_get(khop_server *s, khop_server_counters *out);

/*
 * Change the bound of the worker's wait for a step (the options' 
 * wait_timeout_us; 0 = 2 s) for the steps launched from now on.  A step still
 * running past the bound is given up: the requests it held complete with
 * KHOP_ETIMEDOUT at once, and its slot is reused from zeroed state once the
 * step has finished.  Errors: EINVAL (NULL server, negative bound).
 */
int khop_server_set_wait_timeout(khop_server *s, int64_t wait_timeout_us);

/* Stop the worker; requests not finished are completed with ESHUTDOWN. */
int khop_server_destroy(khop_server *s);

#ifdef __cplusplus
}
#endif

#endif /* KHOP_H */
