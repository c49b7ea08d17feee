/*
 * Plain CPU oracle for single-vertex betweenness in directed graphs.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * statement of what the CUDA library computes. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never calls it and shares no code, header or table with it.
 *
 * Method: Chehreghani, Bifet, Abdessalem, "Exact and Approximate Algorithms
 * for Computing Betweenness Centrality in Directed Graphs".
 *   - Section 2: d(u,v), sigma_st, BC(v) (Eq. 1), the shortest-path DAG (SPD),
 *     dependency delta_s.(v) (Eqs. 2-3) and its recursion (Eq. 4).
 *   - Section 4.1: reverse graph R(G) (Def. 2) and RV(r) by one traversal of
 *     R(G) from r with weights ignored, r excluded (Def. 3, Prop. 2).
 *   - Section 4.2, Algorithm 1 (E-BCD): out-degree test (Prop. 1), RV(r),
 *     then BC(r) = sum over v in RV(r) of delta_v.(r) (Eq. 5).
 *   - Section 4.3, Algorithm 2 (A-BCD): T uniform draws v_t from RV(r),
 *     bc = sum_t delta_{v_t}.(r) * |RV(r)| / T.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Eq. 1 sums ordered pairs s != t; pairs with sigma_st = 0 add nothing.
 *   - sigma is kept exactly (unsigned 128-bit) beside its double value; a
 *     flag is raised when any sigma reaches 2^53, the first count that an
 *     fp64 sum can no longer certify as exact (2^53 + 1 rounds to 2^53).
 *   - Sampling is with replacement. Draw t (t = 0..T-1) takes the first
 *     64-bit word x0 of Philox4x64-10 (Salmon et al., SC'11) with counter
 *     (t, 0, 0, 0) and key (seed, 0), and picks RV index floor(x0*|RV|/2^64)
 *     of the ascending RV list.
 *
 * Everything is fp64 / exact integer arithmetic, sequential per source.
 * Sources are independent (Alg. 1, the loop over RV), so the drivers below
 * may split them over threads; every sum is then taken in a fixed order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

typedef unsigned __int128 u128;

#define ORC_INF UINT64_MAX
#define ORC_FLAG_SIGMA_GT_2_53 1u
#define TWO_POW_53 ((u128)1 << 53)

/* ------------------------------------------------------------------ */
/* Reverse graph R(G), Section 4.1 Def. 2: (u,v) in R(G) iff (v,u) in G. */
/* Counting sort by head; within a row, tails ascend because the forward   */
/* arcs are visited in CSR (ascending tail) order.                          */
/* ------------------------------------------------------------------ */
int orc_reverse(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
                int64_t *roff, int32_t *rcol, uint32_t *rw)
{
    int64_t m = off[n];
    int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cursor) return -1;
    memset(roff, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) roff[col[e] + 1]++;
    for (int32_t v = 0; v < n; v++) roff[v + 1] += roff[v];
    for (int32_t v = 0; v < n; v++) cursor[v] = roff[v];
    for (int32_t u = 0; u < n; u++) {
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            int64_t p = cursor[col[e]]++;
            rcol[p] = u;
            if (w && rw) rw[p] = w[e];
        }
    }
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------ */
/* RV(r), Section 4.1: BFS on R(G) from r, weights ignored; every vertex  */
/* met except r, listed in ascending id. Returns |RV(r)|.                  */
/* ------------------------------------------------------------------ */
int64_t orc_rv(int32_t n, const int64_t *roff, const int32_t *rcol, int32_t r, int32_t *out)
{
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!seen || !queue) { free(seen); free(queue); return -1; }
    int64_t head = 0, tail = 0;
    seen[r] = 1;
    queue[tail++] = r;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int64_t e = roff[x]; e < roff[x + 1]; e++) {
            int32_t y = rcol[e];
            if (!seen[y]) { seen[y] = 1; queue[tail++] = y; }
        }
    }
    int64_t k = 0;
    for (int32_t v = 0; v < n; v++)
        if (seen[v] && v != r) { if (out) out[k] = v; k++; }
    free(seen);
    free(queue);
    return k;
}

/* ------------------------------------------------------------------ */
/* One source: SPD rooted at s (Section 2) and dependencies (Eq. 4).      */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    const int64_t *off, *roff;
    const int32_t *col, *rcol;
    const uint32_t *w, *rw;   /* NULL when unweighted */
} orc_graph;

typedef struct {
    uint64_t *dist;     /* ORC_INF when unreached */
    u128 *sigma_x;      /* exact path counts */
    double *sigma;      /* the same counts in fp64 */
    double *delta;      /* delta_s.(v) */
    int32_t *order;     /* vertices in non-decreasing distance (settle order) */
    int32_t *queue;     /* BFS queue */
    uint64_t *heap_d;   /* Dijkstra heap keys */
    int32_t *heap_v;    /* Dijkstra heap values */
    int64_t heap_cap;
} orc_ws;

static int ws_init(orc_ws *ws, const orc_graph *g)
{
    size_t n = (size_t)g->n;
    memset(ws, 0, sizeof(*ws));
    ws->dist = (uint64_t *)malloc(n * sizeof(uint64_t));
    ws->sigma_x = (u128 *)malloc(n * sizeof(u128));
    ws->sigma = (double *)malloc(n * sizeof(double));
    ws->delta = (double *)malloc(n * sizeof(double));
    ws->order = (int32_t *)malloc(n * sizeof(int32_t));
    ws->queue = (int32_t *)malloc(n * sizeof(int32_t));
    if (g->w) {
        ws->heap_cap = g->off[g->n] + 1;
        ws->heap_d = (uint64_t *)malloc((size_t)ws->heap_cap * sizeof(uint64_t));
        ws->heap_v = (int32_t *)malloc((size_t)ws->heap_cap * sizeof(int32_t));
        if (!ws->heap_d || !ws->heap_v) return -1;
    }
    if (!ws->dist || !ws->sigma_x || !ws->sigma || !ws->delta || !ws->order || !ws->queue) return -1;
    return 0;
}

static void ws_free(orc_ws *ws)
{
    free(ws->dist); free(ws->sigma_x); free(ws->sigma); free(ws->delta);
    free(ws->order); free(ws->queue); free(ws->heap_d); free(ws->heap_v);
}

/* binary min-heap on (key, vertex) with lazy deletion */
static void heap_push(orc_ws *ws, int64_t *size, uint64_t key, int32_t v)
{
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (ws->heap_d[p] <= key) break;
        ws->heap_d[i] = ws->heap_d[p];
        ws->heap_v[i] = ws->heap_v[p];
        i = p;
    }
    ws->heap_d[i] = key;
    ws->heap_v[i] = v;
}

static void heap_pop(orc_ws *ws, int64_t *size, uint64_t *key, int32_t *v)
{
    *key = ws->heap_d[0];
    *v = ws->heap_v[0];
    int64_t last = --(*size);
    uint64_t kd = ws->heap_d[last];
    int32_t kv = ws->heap_v[last];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= last) break;
        if (c + 1 < last && ws->heap_d[c + 1] < ws->heap_d[c]) c++;
        if (ws->heap_d[c] >= kd) break;
        ws->heap_d[i] = ws->heap_d[c];
        ws->heap_v[i] = ws->heap_v[c];
        i = c;
    }
    if (last > 0) { ws->heap_d[i] = kd; ws->heap_v[i] = kv; }
}

/*
 * Distances from s: BFS with a FIFO queue (unweighted; d counts arcs) or
 * Dijkstra with a binary heap (positive integer weights; d sums weights).
 * Fills ws->order with the reached vertices in settle order, returns count.
 */
static int64_t distances(const orc_graph *g, orc_ws *ws, int32_t s)
{
    int32_t n = g->n;
    for (int32_t v = 0; v < n; v++) ws->dist[v] = ORC_INF;
    int64_t k = 0;
    ws->dist[s] = 0;
    if (!g->w) {
        int64_t head = 0, tail = 0;
        ws->queue[tail++] = s;
        while (head < tail) {
            int32_t x = ws->queue[head++];
            ws->order[k++] = x;
            for (int64_t e = g->off[x]; e < g->off[x + 1]; e++) {
                int32_t y = g->col[e];
                if (ws->dist[y] == ORC_INF) {
                    ws->dist[y] = ws->dist[x] + 1;
                    ws->queue[tail++] = y;
                }
            }
        }
    } else {
        uint8_t *done = (uint8_t *)ws->queue; /* reuse as a byte flag array */
        memset(done, 0, (size_t)n);
        int64_t size = 0;
        heap_push(ws, &size, 0, s);
        while (size > 0) {
            uint64_t dx; int32_t x;
            heap_pop(ws, &size, &dx, &x);
            if (done[x] || dx != ws->dist[x]) continue;
            done[x] = 1;
            ws->order[k++] = x;
            for (int64_t e = g->off[x]; e < g->off[x + 1]; e++) {
                int32_t y = g->col[e];
                uint64_t nd = dx + (uint64_t)g->w[e];
                if (nd < ws->dist[y]) {
                    ws->dist[y] = nd;
                    heap_push(ws, &size, nd, y);
                }
            }
        }
    }
    return k;
}

/*
 * Brandes from one source s (Section 2): sigma_sv over the SPD, then the
 * dependencies of Eq. 4, delta_s.(v) = sum_{w : v in P_s(w)} sigma_sv /
 * sigma_sw * (1 + delta_s.(w)). P_s(w) is the set of in-neighbours v of w
 * with d(s,v) + w(v,w) = d(s,w). Returns the flag word.
 */
static unsigned brandes_source(const orc_graph *g, orc_ws *ws, int32_t s, int64_t *reached)
{
    int32_t n = g->n;
    unsigned flags = 0;
    int64_t k = distances(g, ws, s);
    if (reached) *reached = k;
    for (int32_t v = 0; v < n; v++) { ws->sigma_x[v] = 0; ws->sigma[v] = 0.0; ws->delta[v] = 0.0; }
    ws->sigma_x[s] = 1;
    ws->sigma[s] = 1.0;
    /* sigma_sw = sum of sigma_sv over v in P_s(w), in settle order */
    for (int64_t i = 1; i < k; i++) {
        int32_t x = ws->order[i];
        u128 sx = 0;
        double sd = 0.0;
        for (int64_t e = g->roff[x]; e < g->roff[x + 1]; e++) {
            int32_t v = g->rcol[e];
            uint64_t wt = g->rw ? (uint64_t)g->rw[e] : 1u;
            if (ws->dist[v] != ORC_INF && ws->dist[v] + wt == ws->dist[x]) {
                sx += ws->sigma_x[v];
                sd += ws->sigma[v];
            }
        }
        ws->sigma_x[x] = sx;
        ws->sigma[x] = sd;
        if (sx >= TWO_POW_53) flags |= ORC_FLAG_SIGMA_GT_2_53;
    }
    /* Eq. 4, w taken in reverse settle order (deepest first) */
    for (int64_t i = k - 1; i >= 1; i--) {
        int32_t x = ws->order[i];
        double coef = (1.0 + ws->delta[x]);
        for (int64_t e = g->roff[x]; e < g->roff[x + 1]; e++) {
            int32_t v = g->rcol[e];
            uint64_t wt = g->rw ? (uint64_t)g->rw[e] : 1u;
            if (ws->dist[v] != ORC_INF && ws->dist[v] + wt == ws->dist[x])
                ws->delta[v] += ws->sigma[v] / ws->sigma[x] * coef;
        }
    }
    return flags;
}

static void graph_init(orc_graph *g, int32_t n, const int64_t *off, const int32_t *col,
                       const uint32_t *w, const int64_t *roff, const int32_t *rcol, const uint32_t *rw)
{
    g->n = n; g->off = off; g->col = col; g->w = w;
    g->roff = roff; g->rcol = rcol; g->rw = w ? rw : NULL;
}

/*
 * Full single-source state for parity at scale: dist (ORC_INF unreached),
 * sigma (fp64), sigma exact as (lo, hi) 64-bit halves, delta. Any output
 * pointer may be NULL. Returns the flag word, or -1 on allocation failure.
 */
int orc_source_state(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
                     const int64_t *roff, const int32_t *rcol, const uint32_t *rw, int32_t s,
                     uint64_t *dist, double *sigma, uint64_t *sigma_lo, uint64_t *sigma_hi,
                     double *delta, int64_t *reached)
{
    orc_graph g; orc_ws ws;
    graph_init(&g, n, off, col, w, roff, rcol, rw);
    if (ws_init(&ws, &g)) { ws_free(&ws); return -1; }
    unsigned flags = brandes_source(&g, &ws, s, reached);
    for (int32_t v = 0; v < n; v++) {
        if (dist) dist[v] = ws.dist[v];
        if (sigma) sigma[v] = ws.sigma[v];
        if (sigma_lo) sigma_lo[v] = (uint64_t)ws.sigma_x[v];
        if (sigma_hi) sigma_hi[v] = (uint64_t)(ws.sigma_x[v] >> 64);
        if (delta) delta[v] = ws.delta[v];
    }
    ws_free(&ws);
    return (int)flags;
}

/* ------------------------------------------------------------------ */
/* Source loop split over threads; each source's delta_s.(r_q) for every  */
/* query q lands in its own slot, so sums afterwards run in a fixed order. */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_graph *g;
    const int32_t *sources;
    int64_t nsrc;
    const int32_t *queries;
    int32_t nq;
    double *dep;          /* [nsrc][nq]: delta_s.(r_q) */
    unsigned *flags;      /* [nsrc] */
    int64_t *reached;     /* [nsrc] vertices reached from s (may be NULL) */
    int64_t next;         /* shared work counter */
    pthread_mutex_t lock;
    int failed;
} orc_job;

static void *job_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    orc_ws ws;
    if (ws_init(&ws, job->g)) {
        pthread_mutex_lock(&job->lock); job->failed = 1; pthread_mutex_unlock(&job->lock);
        ws_free(&ws);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (i >= job->nsrc) break;
        int64_t reached = 0;
        unsigned f = brandes_source(job->g, &ws, job->sources[i], &reached);
        for (int32_t q = 0; q < job->nq; q++)
            job->dep[i * job->nq + q] = ws.delta[job->queries[q]];
        job->flags[i] = f;
        if (job->reached) job->reached[i] = reached;
    }
    ws_free(&ws);
    return NULL;
}

static int resolve_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/*
 * delta_s.(r_q) for every source in `sources` and every query vertex in
 * `queries` (dep is [nsrc][nq], row-major). flags[i] gets the sigma flag of
 * source i, reached[i] (optional) the number of vertices reached from it.
 */
int orc_dependencies(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
                     const int64_t *roff, const int32_t *rcol, const uint32_t *rw,
                     const int32_t *sources, int64_t nsrc, const int32_t *queries, int32_t nq,
                     double *dep, unsigned *flags, int64_t *reached, int nthreads)
{
    orc_graph g;
    graph_init(&g, n, off, col, w, roff, rcol, rw);
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.g = &g; job.sources = sources; job.nsrc = nsrc;
    job.queries = queries; job.nq = nq; job.dep = dep; job.flags = flags; job.reached = reached;
    pthread_mutex_init(&job.lock, NULL);
    int nt = resolve_threads(nthreads);
    if (nt > nsrc) nt = nsrc > 0 ? (int)nsrc : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, job_worker, &job);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    return job.failed ? -1 : 0;
}

static int64_t out_degree(const int64_t *off, int32_t r) { return off[r + 1] - off[r]; }

/*
 * E-BCD (Algorithm 1): 0 if out-degree(r) = 0 (Prop. 1); otherwise RV(r)
 * by the Section 4.1 procedure and BC(r) = sum_{v in RV(r)} delta_v.(r)
 * (Eq. 5), summed in ascending v. rv_size and flags are optional outputs.
 */
double orc_bc_exact(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
                    const int64_t *roff, const int32_t *rcol, const uint32_t *rw,
                    int32_t r, int nthreads, int64_t *rv_size, unsigned *flags_out)
{
    if (rv_size) *rv_size = 0;
    if (flags_out) *flags_out = 0;
    if (out_degree(off, r) == 0) return 0.0;
    int32_t *rv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t k = orc_rv(n, roff, rcol, r, rv);
    if (rv_size) *rv_size = k;
    double *dep = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    unsigned *fl = (unsigned *)calloc((size_t)(k > 0 ? k : 1), sizeof(unsigned));
    orc_dependencies(n, off, col, w, roff, rcol, rw, rv, k, &r, 1, dep, fl, NULL, nthreads);
    double bc = 0.0;
    unsigned flags = 0;
    for (int64_t i = 0; i < k; i++) { bc += dep[i]; flags |= fl[i]; }
    if (flags_out) *flags_out = flags;
    free(rv); free(dep); free(fl);
    return bc;
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:  */
/* ten rounds of two 64x64->128 multiplies with S-box-free bijection, key   */
/* bumped by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------ */
#define PHILOX_M4x64_0 0xD2E7470EE14C6C93ULL
#define PHILOX_M4x64_1 0xCA5A826395121157ULL
#define PHILOX_W64_0   0x9E3779B97F4A7C15ULL
#define PHILOX_W64_1   0xBB67AE8584CAA73BULL

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        u128 p0 = (u128)PHILOX_M4x64_0 * c0;
        u128 p1 = (u128)PHILOX_M4x64_1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W64_0;
        k1 += PHILOX_W64_1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw t of the sampling stream: an index into an RV list of size k. */
int64_t orc_sample_index(uint64_t seed, int64_t t, int64_t k)
{
    uint64_t ctr[4] = {(uint64_t)t, 0, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return (int64_t)(((u128)out[0] * (u128)(uint64_t)k) >> 64);
}

/*
 * A-BCD (Algorithm 2): 0 if out-degree(r) = 0; RV(r); T draws v_t uniform
 * over RV(r) (with replacement); bc accumulates delta_{v_t}.(r) * |RV| / T
 * in draw order. A source drawn several times is solved once. `samples`
 * (optional, T entries) receives v_t.
 */
double orc_bc_approx(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
                     const int64_t *roff, const int32_t *rcol, const uint32_t *rw,
                     int32_t r, int64_t T, uint64_t seed, int nthreads,
                     int32_t *samples, int64_t *rv_size, unsigned *flags_out)
{
    if (rv_size) *rv_size = 0;
    if (flags_out) *flags_out = 0;
    if (out_degree(off, r) == 0 || T <= 0) return 0.0;
    int32_t *rv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t k = orc_rv(n, roff, rcol, r, rv);
    if (rv_size) *rv_size = k;
    if (k == 0) { free(rv); return 0.0; }
    int32_t *draw = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *uniq = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T < k ? T : k));
    for (int32_t v = 0; v < n; v++) slot[v] = -1;
    int64_t nu = 0;
    for (int64_t t = 0; t < T; t++) {
        int32_t v = rv[orc_sample_index(seed, t, k)];
        draw[t] = v;
        if (samples) samples[t] = v;
        if (slot[v] < 0) { slot[v] = nu; uniq[nu++] = v; }
    }
    double *dep = (double *)malloc(sizeof(double) * (size_t)nu);
    unsigned *fl = (unsigned *)calloc((size_t)nu, sizeof(unsigned));
    orc_dependencies(n, off, col, w, roff, rcol, rw, uniq, nu, &r, 1, dep, fl, NULL, nthreads);
    double bc = 0.0;
    double scale = (double)k / (double)T;
    unsigned flags = 0;
    for (int64_t t = 0; t < T; t++) bc += dep[slot[draw[t]]] * scale;
    for (int64_t i = 0; i < nu; i++) flags |= fl[i];
    if (flags_out) *flags_out = flags;
    free(rv); free(draw); free(slot); free(uniq); free(dep); free(fl);
    return bc;
}

/*
 * Brandes over every source (Section 2, Eq. 3): bc[v] = sum over s != v of
 * delta_s.(v), sources in ascending order. Single-threaded; small graphs.
 */
int orc_bc_all(int32_t n, const int64_t *off, const int32_t *col, const uint32_t *w,
               const int64_t *roff, const int32_t *rcol, const uint32_t *rw, double *bc)
{
    orc_graph g; orc_ws ws;
    graph_init(&g, n, off, col, w, roff, rcol, rw);
    if (ws_init(&ws, &g)) { ws_free(&ws); return -1; }
    unsigned flags = 0;
    for (int32_t v = 0; v < n; v++) bc[v] = 0.0;
    for (int32_t s = 0; s < n; s++) {
        flags |= brandes_source(&g, &ws, s, NULL);
        for (int32_t v = 0; v < n; v++)
            if (v != s) bc[v] += ws.delta[v];
    }
    ws_free(&ws);
    return (int)flags;
}
