/*
 * bcd.h - C ABI of the GB300 library for single-vertex betweenness
 * centrality in directed graphs.
 *
 * Method: Chehreghani, Bifet, Abdessalem, "Exact and Approximate Algorithms
 * for Computing Betweenness Centrality in Directed Graphs".
 *
 *   BC(r)      = sum over ordered pairs s != t, both != r, of sigma_st(r) /
 *                sigma_st (Section 2, Eq. 1); pairs with no path add 0.
 *   RV(r)      = vertices with a path to r, r excluded (Section 4.1, Def. 1),
 *                found by one traversal of the reverse graph R(G) from r with
 *                weights ignored (Def. 2-3, Prop. 2).
 *   E-BCD      = BC(r) = sum over v in RV(r) of delta_v.(r) (Prop. 1, Eq. 5,
 *                Algorithm 1); delta by the recursion of Eq. 4.
 *   A-BCD      = (|RV(r)| / T) * sum over T uniform draws v_t from RV(r) of
 *                delta_{v_t}.(r) (Algorithm 2; Props. 3-4).
 *
 * Conventions for every call:
 *   - Vertex ids are int32 in [0, n). Arcs are directed. A graph has no
 *     self-loops and no repeated arcs (Section 2).
 *   - Scores are raw (not normalised) fp64 sums over ordered pairs.
 *   - Path counts sigma are fp64 integers; when any sigma reaches 2^53 (the
 *     first count an fp64 sum cannot certify as exact) the result carries
 *     BC_FLAG_SIGMA_2_53. That is a flag, not an error.
 *   - Every call runs on the graph's CUDA stream (bc_graph_desc.stream or
 *     bc_set_stream) and returns after its results are in host memory.
 *   - A graph handle may be used by one host thread at a time.
 *   - On failure a call returns a non-zero bc_status and bc_last_error()
 *     gives a message for the calling thread.
 *   - The library allocates and owns its device memory (cudaMalloc); the
 *     caller's arrays are only read during the call.
 */
#ifndef BCD_H
#define BCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BC_OK = 0,
    BC_E_INVALID_ARG = 1,      /* a size, id or parameter out of range */
    BC_E_INVALID_GRAPH = 2,    /* self-loop, repeated or unsorted arc, zero weight */
    BC_E_OOM = 3,              /* device or host allocation failed */
    BC_E_CUDA = 4,             /* a CUDA runtime call failed */
    BC_E_BUFFER_TOO_SMALL = 5, /* output capacity below the needed count */
    BC_E_TIMEOUT = 6,          /* a bounded device wait gave up */
    BC_E_INTERNAL = 7,
    BC_E_BUSY = 8,             /* bc_submit: the server's queue is full; retry later */
    BC_E_PENDING = 9,          /* bc_poll: the query has not finished yet */
    BC_E_CANCELLED = 10        /* bc_cancel stopped the call between two tiles */
} bc_status;

typedef enum { BC_MEM_HOST = 0, BC_MEM_DEVICE = 1 } bc_mem_kind;

/* result flags */
#define BC_FLAG_SIGMA_2_53   0x1u  /* some sigma used for this result is >= 2^53 */
#define BC_FLAG_TRIVIAL_ZERO 0x2u  /* out-degree(r) = 0: BC(r) = 0 by Prop. 1, no traversal */

/*
 * Graph description (Section 2). CSR of the forward graph G:
 *   row_offsets[n+1] int64, non-decreasing, row_offsets[0] = 0,
 *                    row_offsets[n] = m;
 *   cols[m]          int32 heads; within each row strictly increasing
 *                    (sorted, which also rules out repeated arcs), no
 *                    self-loop;
 *   weights[m]       uint32 positive arc lengths of at most 4095 (the
 *                    weighted kernels settle distances in Dial's order
 *                    over a ring of 4096 distance slots), or NULL for an
 *                    unweighted graph (every arc has length 1).
 * mem_kind tells whether the three pointers are host or device memory.
 * stream is a cudaStream_t (NULL: the legacy default stream).
 */
typedef struct {
    int32_t n;
    int64_t m;
    const int64_t *row_offsets;
    const int32_t *cols;
    const uint32_t *weights;
    int32_t mem_kind;
    void *stream;
} bc_graph_desc;

typedef struct bc_graph bc_graph;

/*
 * Copies the graph to the device, validates it and builds the reverse
 * graph R(G) there (Section 4.1, Def. 2). The caller keeps ownership of its
 * arrays. Errors: BC_E_INVALID_ARG (n <= 0, m < 0, NULL pointer, offsets
 * not monotone, head out of range), BC_E_INVALID_GRAPH (self-loop, row not
 * strictly increasing, weight 0 or above 4095), BC_E_OOM, BC_E_CUDA. *out
 * is set only on success.
 */
bc_status bc_graph_create(const bc_graph_desc *desc, bc_graph **out);

/* Frees every device and host resource of the handle. NULL is allowed. */
void bc_graph_destroy(bc_graph *g);

/* Sets the CUDA stream (cudaStream_t) used by later calls on g. */
bc_status bc_set_stream(bc_graph *g, void *stream);

/* n, m and whether the graph carries weights (any pointer may be NULL). */
bc_status bc_graph_info(const bc_graph *g, int32_t *n, int64_t *m, int32_t *weighted);

/*
 * Copies R(G) out to host arrays: roffsets[n+1], rcols[m] and, for a
 * weighted graph, rweights[m] (may be NULL). Row order within a row is
 * unspecified (R(G) is a set of arcs; Def. 2).
 */
bc_status bc_graph_reverse(const bc_graph *g, int64_t *roffsets, int32_t *rcols, uint32_t *rweights);

/*
 * RV(r) (Section 4.1): ids of every vertex with a path to r, r excluded,
 * ascending, written to the host array out[cap]. *count receives |RV(r)|.
 * If cap < |RV(r)| nothing is written and BC_E_BUFFER_TOO_SMALL is
 * returned with *count set (call with out = NULL, cap = 0 to size it).
 */
bc_status bc_rv_compute(bc_graph *g, int32_t r, int32_t *out, int64_t cap, int64_t *count);

/* Per-query report. Times are milliseconds of device work per phase. */
typedef struct {
    int64_t rv_size;          /* |RV(r)| (0 when BC_FLAG_TRIVIAL_ZERO) */
    int64_t samples;          /* T for sampled queries, 0 for exact */
    int64_t sources_run;      /* distinct single-source passes this query used */
    int64_t edges_traversed;  /* sum over those sources s of |E_s|, the arcs whose
                                 tail s reaches (forward pass, counted once) */
    int32_t max_level;        /* deepest SPD level met (unweighted) */
    uint32_t flags;           /* BC_FLAG_* */
    double ms_rv, ms_sample, ms_spd, ms_total;
} bc_info;

/*
 * E-BCD (Algorithm 1): exact BC(r). Zero without any traversal when
 * out-degree(r) = 0 (Prop. 1). info may be NULL.
 */
bc_status bc_exact(bc_graph *g, int32_t r, double *bc, bc_info *info);

/*
 * A-BCD (Algorithm 2) with T = ceil(ln(2/delta) / (2 eps^2)) samples, i.e.
 * Eq. "samplesnumber" with eps relative to the range K*|RV(r)| of one
 * estimate (then |bc - BC(r)| <= eps*K*|RV(r)| with probability >=
 * 1 - delta, Prop. 4). Requires eps > 0 and 0 < delta < 1.
 * Draw t (t = 0..T-1) is RV index floor(x0 * |RV(r)| / 2^64) of the
 * ascending RV(r) list, x0 the first word of Philox4x64-10 with counter
 * (t, 0, 0, 0) and key (seed, 0). Sampling is with replacement.
 */
bc_status bc_approx(bc_graph *g, int32_t r, double eps, double delta, uint64_t seed,
                    double *bc, bc_info *info);

/* A-BCD with an explicit sample count T >= 1 (the paper's fixed tau runs). */
bc_status bc_approx_T(bc_graph *g, int32_t r, int64_t T, uint64_t seed, double *bc, bc_info *info);

/* T for (eps, delta) as bc_approx computes it. */
bc_status bc_samples_for(double eps, double delta, int64_t *T);

/*
 * The T draws v_t of bc_approx_T(r, T, seed), in draw order, written to
 * the host array out[T]; *rv_size receives |RV(r)|. When out-degree(r) = 0
 * or RV(r) is empty no draw is made and *rv_size is 0.
 */
bc_status bc_draw_samples(bc_graph *g, int32_t r, int64_t T, uint64_t seed, int32_t *out,
                          int64_t *rv_size);

typedef enum {
    BC_QUERY_EXACT = 0,     /* Algorithm 1 */
    BC_QUERY_APPROX = 1,    /* Algorithm 2, T from (eps, delta) */
    BC_QUERY_APPROX_T = 2,  /* Algorithm 2, T given */
    BC_QUERY_HYBRID = 3     /* Section 5 procedure: exact if |RV(r)| <= T, else
                               Algorithm 2 with T samples */
} bc_query_kind;

typedef struct {
    int32_t r;
    int32_t kind;     /* bc_query_kind */
    double eps;       /* APPROX */
    double delta;     /* APPROX */
    int64_t T;        /* APPROX_T, HYBRID (tau) */
    uint64_t seed;    /* APPROX, APPROX_T, HYBRID */
} bc_query;

typedef struct {
    double bc;
    int32_t status;   /* bc_status of this query */
    uint32_t flags;   /* BC_FLAG_* */
    int64_t rv_size;
    int64_t samples;  /* T used (0 for an exact answer) */
} bc_result;

typedef struct {
    int64_t queries;
    int64_t sources_run;      /* distinct sources over all queries (set version,
                                 Section 4.2: one SPD per vertex of the union) */
    int64_t edges_traversed;  /* sum over those sources of |E_s| */
    int64_t launches;         /* kernel launches issued */
    double ms_rv, ms_sample, ms_spd, ms_total;
    double ms_forward;        /* wall time of the traversal kernel's forward */
    double ms_backward;       /* ... and backward passes (one block's view) */
    int64_t tiles;            /* tiles run (64*tile_words sources each; 64*weighted_words on weighted graphs) */
    int32_t max_level;        /* deepest SPD level met */
    int32_t grid_blocks;      /* blocks of the persistent traversal launch */
    double ms_traversal;      /* CUDA-event time of the batched traversal launches */
    int64_t reached_pairs;    /* sum over sources s of |V_s| (vertices s reaches) */
    int64_t tight_pairs;      /* sum over sources s of the arcs of s's SPD (weighted
                                 source kernel: the sigma offers that took effect, which
                                 also counts ties a shorter path later replaced) */
    int64_t arc_visits;       /* arcs scanned by the traversal, both passes */
    int64_t union_vertices;   /* sum over tiles of vertices any tile source reaches
                                 (weighted source kernel: over each launch) */
    int64_t union_arcs;       /* sum over tiles of the out-arcs of those vertices */
    int64_t scan_pairs;       /* accumulation 2: (t, s) pairs with the query vertex on a
                                 shortest s-t path (the terms of the vertex scan) */
    double ms_root;           /* accumulation 2: CUDA-event time of the traversal from the
                                 query vertex (inside ms_spd, not in ms_traversal) */
    int64_t pull_levels;      /* forward levels run bottom-up (bc_config.pull_permille) */
    int64_t scan_tiles;       /* tiles whose dependencies came from the vertex scan */
    int64_t eq4_reached_pairs; /* reached_pairs and tight_pairs of the tiles that ran the */
    int64_t eq4_tight_pairs;   /* backward pass of Eq. 4 (the others ran the vertex scan) */
} bc_batch_info;

/*
 * Many queries at once (the set version of Section 4.2): one RV traversal
 * per group of up to 64 queries, then one single-source pass per vertex of
 * the union of their source sets, shared by every query that needs it.
 * out[nq] receives one result per query, each identical (within fp64
 * summation order) to the single-query call. Returns BC_OK when every
 * query was attempted; per-query failures are in out[i].status.
 * info may be NULL.
 */
bc_status bc_batch(bc_graph *g, const bc_query *queries, int64_t nq, bc_result *out,
                   bc_batch_info *info);

/*
 * One shard of bc_batch, for spreading a batch over several GPUs (one
 * process and one graph replica per GPU): the sources of a group are
 * independent terms of the sums of Algorithm 1 and 2 (and of the set version
 * of Section 4.2), so shard k of nshards runs only tiles [T*k/nshards,
 * T*(k+1)/nshards) of each group's T tiles, in the order bc_batch runs them,
 * and out[i].bc receives that shard's part of query i's score (scaled by
 * |RV(r)|/T for sampled queries). The scores of shards 0 .. nshards-1 add up
 * to the bc_batch score (equal up to fp64 summation order); rv_size, samples
 * and status are the same on every shard, and flags are to be OR-ed.
 * Requires 0 <= shard < nshards, else BC_E_INVALID_ARG. nshards = 1 is
 * bc_batch.
 */
bc_status bc_batch_shard(bc_graph *g, const bc_query *queries, int64_t nq, int32_t shard, int32_t nshards,
                         bc_result *out, bc_batch_info *info);

/*
 * Parity probe: runs the single-source passes for 1 .. 64*w distinct
 * sources (one tile of the batched kernel, w = tile_words on unweighted
 * graphs, weighted_words on weighted ones; more is BC_E_INVALID_ARG) and
 * returns, for each source
 * i and vertex v, dist[i*n + v] (UINT64_MAX when unreached; hop count for
 * an unweighted graph) and sigma[i*n + v] (fp64), and for each target
 * vertex t_j, dep[i*nt + j] = delta_{s_i}.(t_j) (Eq. 4). Any output may be
 * NULL. flags (may be NULL) receives BC_FLAG_SIGMA_2_53 per source.
 * Host arrays.
 */
bc_status bc_spd_probe(bc_graph *g, const int32_t *sources, int32_t nsrc, const int32_t *targets,
                       int32_t nt, uint64_t *dist, double *sigma, double *dep, uint32_t *flags);

/*
 * Serving with continuous batching (the set version of Section 4.2 applied to
 * a stream of queries). A server owns a worker thread that runs queries on
 * the graph; while it exists, the graph must not be used by other calls.
 *
 * Admission: a submitted query waits until one of max_active query slots
 * (at most 64) is free. Then its source set is prepared (RV(r); Philox draws
 * for sampled queries) and it is admitted while the device bytes that its
 * distinct sources hold until they have run (12 bytes each, 268 for a
 * sampled query, which also stages its draw counts, plus 512 per tile of
 * partial sums), added to those of the queries already admitted, stay within
 * max_device_bytes; otherwise it returns to the head of the queue until
 * running queries free their bytes, and a query whose bytes alone exceed the
 * budget completes with status BC_E_BUSY. The per-(vertex, source) slabs
 * (sigma, accumulators, masks, level history) are allocated once per graph
 * for one tile and shared by all tiles, outside the budget. An admitted
 * query's sources join the pool of pending sources: a source already pending
 * for another query is run once for both. The worker runs the pool in slices
 * of tiles_per_slice tiles, taking sources round-robin across the active
 * queries, so queries that arrive while others run get their work into the
 * next slice. Each result equals the single-query call up to fp64 summation
 * order.
 */
typedef struct bc_server bc_server;

typedef struct {
    int32_t max_active;          /* query slots in flight, 1..64 (0: 64) */
    int32_t tiles_per_slice;     /* tiles per traversal launch (0: 16) */
    int64_t max_device_bytes;    /* admission budget in device bytes (0: a quarter of the
                                    free device memory at bc_server_create) */
    int64_t max_queue;           /* bound on submitted, unadmitted queries (0: 2^20) */
} bc_server_config;

typedef struct {
    int64_t submitted, admitted, completed;
    int64_t slices;              /* traversal launches */
    int64_t sources_run;
    int64_t edges_traversed;
    int64_t active, queued;      /* at the time of the call */
    double busy_ms;              /* wall time of the slices */
} bc_server_stats;

/* Starts the worker. cfg may be NULL (defaults). */
bc_status bc_server_create(bc_graph *g, const bc_server_config *cfg, bc_server **out);

/* Queues a query; *ticket identifies it. BC_E_BUSY when the queue is full,
 * BC_E_INVALID_ARG for a bad query (no ticket then). Thread-safe. */
bc_status bc_submit(bc_server *srv, const bc_query *q, uint64_t *ticket);

/* Waits up to timeout_us for the query; BC_OK fills *out (and the latency
 * from submission to completion, if latency_ms is not NULL) and releases the
 * ticket; BC_E_PENDING if not finished yet. Thread-safe. */
bc_status bc_poll(bc_server *srv, uint64_t ticket, bc_result *out, double *latency_ms, int64_t timeout_us);

bc_status bc_server_stats_get(bc_server *srv, bc_server_stats *stats);

/* Stops the worker (unfinished queries are dropped) and frees the server. */
void bc_server_destroy(bc_server *srv);

/*
 * Tuning of the batched traversal (no effect on results beyond fp64
 * summation order of delta):
 *   tile_words     mask words per tile: 1, 2, 4 or 8 (64, 128, 256 or 512
 *                  sources advanced together; bc_graph_create picks the
 *                  widest of 1, 2 and 4 whose sigma and accumulator slabs,
 *                  16 bytes per (vertex, source) pair, fit in half of the
 *                  free device memory; 8 runs one block per SM);
 *   chunk_arcs     arcs per unit of work when a vertex's row is split
 *                  (32..65536, a multiple of 32);
 *   block_threads  threads per block of the persistent kernel (128..512,
 *                  a multiple of 32; on unweighted graphs at least
 *                  64 * tile_words, else BC_E_INVALID_ARG);
 *   source_order   how the union of sources is cut into tiles: 1 (default)
 *                  sorts sources by their hop distance to the vertex of
 *                  largest in-degree x out-degree, then by the number of
 *                  arcs two hops away (largest first), so that a tile's BFS
 *                  levels line up;
 *                  2 keeps ascending vertex ids;
 *   blocks_per_sm  resident blocks per SM for tile_words = 4 (1 or 2; 2,
 *                  the default, trades register spills for occupancy);
 *   weighted_words sources per tile of the weighted tile kernel, in words
 *                  of 64 (1, 2, 4, 8 or 16, with n * 64 * weighted_words <=
 *                  2^32); on the source kernel only the grouping of the
 *                  per-query partial sums.
 *                  bc_graph_create picks 4, or less when that does not fit
 *                  in half of the free device memory at about 40 bytes per
 *                  (vertex, source) pair. tile_words applies to unweighted
 *                  graphs only.
 *   accumulation   how the dependencies delta_s.(r) of a launch are summed:
 *                  1 the backward pass of Eq. 4, deepest level first
 *                  (unweighted: pushed along the tight in-arcs of R(G);
 *                  weighted: pulled over the tight out-arcs);
 *                  2 a vertex scan when every query of a call (or of a
 *                  bc_batch group) has the same vertex r, else 1: one
 *                  forward traversal from r gives d(r,t) and sigma_rt, and
 *                  after each tile's forward pass
 *                    delta_s.(r) = sigma_sr * sum over t != s, r with
 *                                  d(s,r) + d(r,t) = d(s,t) of sigma_rt / sigma_st
 *                  (Eq. 2 summed over the pair dependencies, with
 *                  sigma_st(r) = sigma_sr * sigma_rt when r lies on a
 *                  shortest s-t path: the Bellman criterion), one pass over
 *                  the tile's reached (vertex, source) pairs with no
 *                  per-level barrier, on unweighted and weighted graphs;
 *                  3 the vertex scan for every group, with its queries at
 *                  up to 64 distinct vertices r_c: one traversal rooted at
 *                  all of them gives d(r_c, t) and sigma_{r_c t} (12 bytes
 *                  per vertex and column on unweighted graphs, 16 on
 *                  weighted ones; 64 columns allocated on first use), and
 *                  each tile's pass (each source's, on the weighted source
 *                  kernel) screens its reached (vertex, source) pairs for
 *                  the columns of the queries that need the source;
 *                  4 (default) 2 for one-vertex groups and, for a group
 *                  at several vertices, 3 on its
 *                  first tile, then for the remaining tiles the scan when
 *                  its terms on that tile, weighted 16 to 1, did not
 *                  outnumber the tight (source, arc) pairs the Eq. 4 push
 *                  would add, else 1. The scan wins where few shortest
 *                  paths run through the query vertices (1.5x on the
 *                  benchmark's R-MAT 22 batch of 64 uniform vertices) and
 *                  loses on hubs (4-5x slower for the 32 vertices of
 *                  largest in-degree x out-degree of R-MAT 20).
 *                  Results equal those of 1 up to fp64 rounding order.
 *   pull_permille  direction of each forward level of the unweighted kernel:
 *                  a level whose frontier's out-arcs number at least
 *                  pull_permille / 1000 of the graph's arcs runs bottom-up
 *                  (every vertex not yet reached by some source of the tile
 *                  scans its in-arcs in R(G) and sums sigma over the
 *                  in-neighbours on the current level, with no atomic per
 *                  arc), the others top-down (the frontier pushes sigma
 *                  along its out-arcs); 1..1000, or -1 for top-down only.
 *                  Results are identical either way (sigma sums integers).
 *   weighted_short_row  weighted kernels: a settled vertex (source kernel:
 *                  whose out-row; tile kernel: a (vertex, source) pair whose
 *                  in- and out-rows both) has at most this many arcs is
 *                  handled by the lanes given to it in its level (1 to 32,
 *                  tile kernel 1 to 8); longer rows are cut into chunk_arcs
 *                  chunks that a warp takes with lanes over arcs (1..1024,
 *                  default 32).
 *   timeout_us     limit, in microseconds of wall time, on every wait of a
 *                  traversal kernel at a grid-wide barrier (default
 *                  10,000,000: 10 s), and on the time one block of the
 *                  weighted source kernel spends on one source. A wait or a
 *                  source that runs out makes every block leave the kernel;
 *                  the call returns BC_E_TIMEOUT, the graph's device state
 *                  is reset and the handle stays usable.
 *   weighted_kernel  organisation of the weighted SPD: 1 the tile kernel
 *                  (the 64 * weighted_words sources of a tile settle their
 *                  (vertex, source) pairs together, one grid-wide barrier
 *                  per distance value); 2 (default) the source kernel: each
 *                  block (1024 threads, one per SM; block_threads does not
 *                  apply) takes one source at a time and settles its
 *                  distances with block barriers only, so blocks never wait
 *                  on one another (per block: 20 bytes per vertex plus the
 *                  bucket ring; as many blocks as fit in half of the free
 *                  device memory, up to one per SM). Both give
 *                  the same distances and sigma; dependencies agree up to
 *                  fp64 summation order. The traversal rooted at the query
 *                  vertices of the vertex scan, and bc_spd_probe, always
 *                  run on the tile kernel.
 * Zero fields keep their current value.
 */
typedef struct {
    int32_t tile_words;
    int32_t chunk_arcs;
    int32_t block_threads;
    int32_t source_order;
    int32_t blocks_per_sm;
    int32_t weighted_words;
    int32_t accumulation;
    int32_t timeout_us;
    int32_t pull_permille;
    int32_t weighted_short_row;
    int32_t weighted_kernel;
} bc_config;

bc_status bc_set_config(bc_graph *g, const bc_config *cfg);
bc_status bc_get_config(const bc_graph *g, bc_config *cfg);

/*
 * Autotuner of the batched traversal's launch parameters for a graph and a
 * kind of batch. The probe batch is queries[0 .. min(nq, 64)) with every
 * query turned into A-BCD with min(T, probe_T) draws (same vertices and
 * seeds), so each candidate costs a few tiles. Starting from the graph's
 * current configuration, one parameter at a time takes each of its
 * candidate values with the others fixed, and the fastest (CUDA-event time
 * of the batch, second of two runs) is kept:
 *   unweighted: tile_words 2, 4, 8; blocks_per_sm 1, 2; chunk_arcs 64, 128, 256;
 *               pull_permille -1, 200; accumulation 1, 4;
 *   weighted:   weighted_kernel 1, 2; weighted_words 2, 4, 8;
 *               weighted_short_row 16, 32, 64; chunk_arcs 64, 128, 256;
 *               accumulation 1, 4.
 * Candidates that do not fit in device memory are skipped. The winner is
 * applied to g and written to *best; rep (may be NULL) receives the number
 * of candidates timed and the probe times of the starting and the chosen
 * configuration. Results of later calls are unchanged beyond fp64 summation
 * order. Errors: BC_E_INVALID_ARG (nq < 1, probe_T outside 1..10^6), and
 * those of bc_batch (the starting configuration is restored).
 */
typedef struct {
    int64_t candidates;     /* configurations timed */
    int64_t probe_queries;  /* queries in the probe batch */
    double ms_default;      /* probe time of the starting configuration */
    double ms_best;         /* probe time of the chosen one */
} bc_tune_report;

bc_status bc_tune(bc_graph *g, const bc_query *queries, int64_t nq, int64_t probe_T, bc_config *best,
                  bc_tune_report *rep);

/*
 * RV(r) for callers that cannot allocate device memory. (The paper has no
 * counterpart: this is a deployment variant of bc_rv_compute.)
 *
 * Some callers may not call cudaMalloc: code running inside another
 * framework's allocator callbacks or teardown, processes whose device memory
 * is fully reserved by a caching allocator, and plugins that are handed a
 * stream and caller-owned buffers but no right to allocate. This call
 * allocates nothing. Its working memory is one file-scope device array of
 * about 33 MB (a visited bitmap and two frontier queues sized for
 * BC_NOALLOC_MAX_VERTICES vertices), which every GPU that loads the library
 * holds until the process exits.
 *
 *   d_roffsets[n+1], d_rcols[m]  R(G) in CSR form, device memory (for example
 *                                from bc_graph_reverse, copied back to the
 *                                device by the caller); weights are not used;
 *   n                            1 .. BC_NOALLOC_MAX_VERTICES, else
 *                                BC_E_INVALID_ARG;
 *   r                            the query vertex;
 *   d_out[cap]                   device buffer for RV(r), ascending, r
 *                                excluded; nothing is written when
 *                                cap < |RV(r)| (BC_E_BUFFER_TOO_SMALL);
 *   *count                       host: |RV(r)|;
 *   stream                       cudaStream_t the work is queued on; the call
 *                                returns after it has finished.
 *
 * The first call on a device looks up the array's device address (and may
 * load the module there); make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents; the
 * call clears what must start empty. Calls that overlap on the GPU (from two
 * threads or two streams) race on the array and must be serialised by the
 * caller.
 */
#define BC_NOALLOC_MAX_VERTICES 4194304
bc_status bc_rv_compute_noalloc(const int64_t *d_roffsets, const int32_t *d_rcols, int32_t n, int32_t r,
                                int32_t *d_out, int64_t cap, int64_t *count, void *stream);

/*
 * Cancels the call that is running on g (from another host thread; the one
 * call that may overlap another on the same handle). The traversal kernels
 * read the request when a tile of sources starts, so the running call stops
 * within one tile, resets the graph's device state and returns
 * BC_E_CANCELLED (bc_batch: every query of the stopped group gets that
 * status). A request made while no call runs is dropped when the next call
 * starts. The handle stays usable.
 */
bc_status bc_cancel(bc_graph *g);

/*
 * Fault injection on the host, for tests of the error paths: the k-th
 * device allocation the library makes from now on (k >= 1, counted over all
 * handles of the process) fails as if cudaMalloc had returned an
 * out-of-memory error, so that call returns BC_E_OOM; k = 0 switches the
 * injection off. A call that fails this way frees the handle's working
 * memory, which the next call allocates again; the graph stays usable.
 * k < 0 is BC_E_INVALID_ARG.
 */
bc_status bc_debug_fail_alloc(int64_t k);

/* Message for the last failed call on this thread ("" if none). */
const char *bc_last_error(void);

/* Version string of the library. */
const char *bc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BCD_H */
