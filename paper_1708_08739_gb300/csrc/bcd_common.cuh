// Internal declarations shared by the CUDA translation units of libbcd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bcd.h"

namespace bcd {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// device error codes written to Counters::err
enum DevErr : int32_t {
    kDevOk = 0,
    kDevHistOverflow = 1,
    kDevChunkOverflow = 2,
    kDevTimeout = 4,
    kDevLevelOverflow = 5,
    kDevBucketOverflow = 6,
    kDevCancelled = 7,
    kDevWide = 8,  // weighted source kernel: a count or distance needs the 16-byte pairs
};

// Per-launch control block of the persistent traversal kernel.
struct Counters {
    int32_t err;
    uint32_t bar_count;
    uint32_t bar_gen;
    uint32_t pad0;
    unsigned long long edges;      // sum over reached (v, s) of out-degree(v)
    unsigned long long levels_max; // deepest level met over all tiles
    unsigned long long ns_fwd;     // block 0's wall time in forward passes
    unsigned long long ns_bwd;     // ... in backward passes
    unsigned long long ns_other;   // ... in tile set-up and tear-down
    unsigned long long reached;    // sum over sources s of |V_s| (vertices s reaches, s included)
    unsigned long long tight;      // sum over sources s of tight arcs (sigma additions)
    unsigned long long arc_visits; // arcs scanned, forward plus backward
    unsigned long long vb;         // sum over tiles of distinct vertices reached
    unsigned long long eb;         // sum over tiles of the out-arcs of those vertices
    unsigned long long vpairs;     // vertex scan: (t, s) pairs with the query vertex on a shortest s-t path
    unsigned long long pull_levels; // forward levels run bottom-up (pull over R(G))
};

// One unit of expansion work: arcs [a0, a0 + na) of vertex v, the k-th of
// nch chunks of history entry e.
struct __align__(16) Chunk {
    int32_t v;
    int32_t e;
    int32_t k;
    int32_t nch;
    int64_t a0;
    int32_t na;
    int32_t pad;   // unweighted out-arc chunks: the row's length; weighted: kind (0 out, 1 in) | source << 1
};

// Traversal modes of the persistent kernel.
enum TravMode : int32_t {
    kModeReach = 0,  // masks only (RV on R(G)); no sigma, no backward
    kModeSpd = 1,    // sigma forward, dependency backward (Eq. 4)
    kModeScan = 2,   // sigma forward, dependencies on one query vertex by a vertex scan
};

// Flags of a traversal launch.
enum TravFlags : int32_t {
    kFlagNoBackward = 1,   // stop after the forward pass
    kFlagNoReset = 2,      // leave the dense state dirty (probe export)
    kFlagFullBackward = 4, // backward down to level 0 for every source
    kFlagRootOut = 8,      // scan mode: write the level and sigma of source slot 0 to rlev / rsig
};

struct TravParams {
    int32_t n;
    int32_t mode;
    int32_t flags;
    int32_t chunk_arcs;
    const int64_t *off;
    const int32_t *col;
    // dense per-vertex state
    uint64_t *vs;       // [n * vs_stride]: vis[W], dm0[W], dm1[W] (+pad)
    int32_t vs_stride;  // words per vertex
    int32_t pad0;
    int32_t *tag;       // [n] last level a vertex was appended at, -1 none
    double *sigma;      // [n * S] sigma, then c = (1 + delta) / sigma in place
    double *acc;        // [n * S] backward sums of c over tight out-arcs (unweighted), zero between levels
    // level history
    int32_t *hv;        // [hcap]
    uint64_t *hm;       // [hcap * W] (unweighted)
    uint16_t *hs;       // [hcap] source slot of an entry (weighted)
    int64_t hcap;
    Chunk *chunks;      // [ccap]
    Chunk *ichunks;     // [ccap] in-arc (R(G)) chunks of the entries, per level (unweighted SPD)
    int64_t ccap;
    double *partial;    // [pcap * S]
    int32_t *pdone;     // [pcap]
    int64_t pcap;
    unsigned long long *lev_cnt;   // [maxlev + 2]
    unsigned long long *lev_ccnt;  // [maxlev + 2]
    unsigned long long *lev_grab;  // [2 * (maxlev + 2)] chunk hand-out counters, forward then backward
    int64_t *lev_start;            // [maxlev + 2]
    int64_t *lev_cstart;           // [maxlev + 2]
    int64_t *lev_icstart;          // [maxlev + 2] first in-arc chunk of each level
    int32_t maxlev;
    int32_t pad1;
    // bottom-up forward levels: every vertex's in-arcs (R(G)) in chunks of
    // chunk_arcs, as (vertex, chunk index) pairs, and the switch: a level runs
    // bottom-up when its frontier's out-arcs reach pull_arcs_min (0: never)
    const int2 *pchunks;
    int64_t npchunks;
    int64_t pull_arcs_min;
    // tiles
    const int32_t *srcs;  // [ntiles * S], -1 pads the last tile
    int64_t ntiles;
    // queries (SPD mode); a group holds at most 64 queries (one mask word)
    const uint64_t *qmask;   // [n] bit q set at vertex r_q
    const uint64_t *need;    // [n] bit q set when query q uses the vertex as a source
    uint64_t exact_q;        // queries whose multiplicity is the need bit
    const uint32_t *mult;    // [ntiles * S * 64] draw counts of sampled queries, or NULL
    int32_t *qlevel;         // [S * 64]
    double *dep;             // [S * 64]
    double *tile_partial;    // [ntiles * 64]
    uint32_t *qflags;        // [64]
    uint64_t *srcflag;       // [W] sigma >= 2^53 seen for a source slot (this tile)
    // weighted graphs (Dial buckets on exact distances)
    const uint32_t *wt;      // [m] forward arc weights
    const int64_t *roff;     // [n + 1] R(G)
    const int32_t *rcol;     // [m]
    const uint32_t *rwt;     // [m] weights of R(G)'s arcs
    uint64_t *dist;          // [n * S] tentative, then final distances (UINT64_MAX unreached)
    uint32_t *buckets;       // [ring * bcap] queued pairs (vertex << log2 S | source slot), circular per slot
    unsigned long long *bcount;  // [2 * ring] entries ever queued per slot, then entries consumed per slot
    int64_t bcap;            // entries per slot (a power of two)
    int32_t ring;            // power of two above the largest weight
    int32_t nw;              // 64-source words of a weighted tile (1, 2, 4, 8 or 16)
    int32_t wshort;          // weighted: rows of at most this many arcs are walked by one lane
    int64_t *lev_dist;       // [maxlev + 2] distance of each non-empty level
    // vertex scan (one query vertex vroot): its forward traversal and per-source sums
    int32_t *rlev;           // [n] d(vroot, t), -1 unreached (unweighted)
    uint64_t *rdist;         // [n] d(vroot, t), UINT64_MAX unreached (weighted)
    double *rsig;            // [n] sigma from vroot to t
    double *vsum;            // [2 S] per-source sums of the current tile (unweighted: sigma_sr * sum_t
                             // sigma_rt / sigma_st; weighted: sum_t sigma_rt / sigma_st, then sigma_sr)
    int32_t vroot;
    int32_t pad2;
    // vertex scan over several query vertices (columns): column c of the
    // group's distinct query vertices croot[c]; query bit q belongs to column
    // qcol[q]; rlevq / rsigq [t * 64 + c] = d(croot[c], t) and sigma from it
    // (weighted: rdistq / rsigq [t * wcols_stride(ncols) + c]);
    // msum [s * 64 + c] the per-(source, column) sums of the current tile
    int32_t ncols;           // 0 or 1: the one-vertex scan above
    int32_t pad3;
    const int32_t *qcol;     // [64]
    const int32_t *croot;    // [64]
    int32_t *rlevq;          // [n * 64], -1 unreached (unweighted)
    uint64_t *rdistq;        // [n * 64] allocated, UINT64_MAX unreached (weighted)
    double *rsigq;           // [n * 64]
    double *msum;            // [2 * S * 64]: sums, then (weighted) sigma_s(croot[c])
    // reach mode output
    uint64_t *rvmask;        // [n]
    int32_t *levout;         // [n] level of first discovery (reach mode, one root), or NULL
    Counters *ctr;
    double timeout_ns;
    const int32_t *cancel;   // host-mapped flag, non-zero: leave at the next tile start (may be NULL)
};

}  // namespace bcd

// ---------------------------------------------------------------------------
// Library internals shared across translation units
// ---------------------------------------------------------------------------

struct bcd_workspace {
    int W = 0;           // mask words per tile (S = 64 W sources)
    int64_t n = 0;
    int64_t m = 0;
    // dense state
    uint64_t *vs = nullptr;
    int vs_stride = 0;
    int32_t *tag = nullptr;
    double *sigma = nullptr;
    double *acc = nullptr;        // [n * 64 * W] unweighted graphs
    // history
    int32_t *hv = nullptr;
    uint64_t *hm = nullptr;
    int64_t hmcap = 0;            // entries hm holds (hcap but on weighted graphs)
    uint16_t *hs = nullptr;
    int64_t hcap = 0;
    bcd::Chunk *chunks = nullptr;
    bcd::Chunk *ichunks = nullptr;
    int64_t ccap = 0;
    double *partial = nullptr;
    int32_t *pdone = nullptr;
    int64_t pcap = 0;
    unsigned long long *lev_cnt = nullptr;
    unsigned long long *lev_ccnt = nullptr;
    unsigned long long *lev_grab = nullptr;  // [6 * (maxlev + 2)]: forward and backward hand-out, in-arc chunk
                                             // counts, frontier out-arc sums, entries | chunks << 32
    int64_t *lev_start = nullptr;
    int64_t *lev_cstart = nullptr;
    int64_t *lev_icstart = nullptr;
    int32_t maxlev = 0;
    int2 *pchunks = nullptr;      // in-arc chunks of every vertex (bottom-up levels), unweighted graphs
    int64_t npchunks = 0;
    int32_t pchunk_arcs = 0;      // chunk_arcs the list was cut with
    // per-group state
    uint64_t *rvmask = nullptr;   // [n]
    uint64_t *need = nullptr;     // [n]
    uint64_t *qmask = nullptr;    // [n]
    int32_t *posd = nullptr;      // [n] position of a vertex in the source union
    int32_t *hublev = nullptr;    // [n] hop distance to the hub (tile ordering key), -1 unreached
    // weighted graphs
    uint64_t *dist = nullptr;     // [n * 64 * W]
    uint32_t *buckets = nullptr;  // [ring * bcap]
    unsigned long long *bcount = nullptr;  // [2 * ring]
    int64_t bcap = 0;
    int64_t *lev_dist = nullptr;  // [maxlev + 2]
    int32_t ring = 0;
    int32_t hub = -1;             // vertex the ordering key is measured to
    int32_t *dlist = nullptr;     // [n + 64 * W + 256] source union, padded to whole tiles
    int32_t *qlevel = nullptr;    // [64 * W * 64]
    double *dep = nullptr;        // [64 * W * 64]
    int32_t *rlev = nullptr;      // [n] vertex scan: levels from the query vertex (unweighted graphs)
    uint64_t *rdist = nullptr;    // [n] ... distances from it (weighted graphs)
    double *rsig = nullptr;       // [n] ... and its path counts
    double *vsum = nullptr;       // [2 * 64 * W] ... and the per-source sums of a tile
    int32_t *rlevq = nullptr;     // [n * 64] several query vertices: levels from each (unweighted graphs)
    uint64_t *rdistq = nullptr;   // [n * 64] ... distances from each (weighted graphs)
    double *rsigq = nullptr;      // [n * 64] ... and path counts
    double *msum = nullptr;       // [64 * W * 64] per-(source, column) sums of a tile
    int32_t *rtile = nullptr;     // [64 * W] the one-source tile of the query vertex's traversal
    uint32_t *qflags = nullptr;   // [64]
    uint64_t *srcflag = nullptr;  // [W]
    // weighted source kernel (one source per block): per-block state
    int32_t sblocks = 0;                   // blocks the state is sized for
    unsigned long long *sds = nullptr;     // [sblocks * n * 2]: (distance, sigma) of each vertex
    uint32_t *stb = nullptr;               // [sblocks * (m + 31) / 32]: tight-candidate arc bits
    int32_t slayout = 0;                   // how sds is cleared: 1 16-byte pairs, 2 8-byte words
    bool swide = false;                    // a narrow launch overflowed: 16-byte pairs from now on
    int32_t *shv = nullptr;                // [sblocks * n]
    int32_t *slstart = nullptr;            // [sblocks * smaxlev]
    unsigned long long *sldist = nullptr;  // [sblocks * smaxlev]
    uint32_t *sbk = nullptr;               // [sblocks * ring * sbcap]
    bcd::Chunk *sch = nullptr;             // [sblocks * schcap]
    double *spart = nullptr;               // [sblocks * schcap]
    int64_t sbcap = 0;
    int64_t schcap = 0;
    int32_t smaxlev = 0;
    double *sdep = nullptr;                // [sources * 64] per-source dependencies
    int64_t sdep_cap = 0;
    uint32_t *sflag = nullptr;             // [sources]
    int64_t sflag_cap = 0;
    unsigned long long *snext = nullptr;   // source hand-out counter
    bcd::Counters *ctr = nullptr;
    int64_t *scratch64 = nullptr; // [scratch_len + 256] scan/compaction scratch, counts past scratch_len
    int64_t scratch_len = 0;
    uint64_t *small = nullptr;    // [kSmallWords] tables staged from the host for one group
    // growable
    double *tile_partial = nullptr;
    int64_t tile_partial_cap = 0;
    uint32_t *mult = nullptr;
    int64_t mult_cap = 0;
    int32_t *rvlists = nullptr;
    int64_t rvlists_cap = 0;
    int32_t *draws = nullptr;
    int64_t draws_cap = 0;
    int64_t *blocksums = nullptr;
    int64_t blocksums_cap = 0;
    // host pinned staging
    void *pinned = nullptr;
    size_t pinned_cap = 0;
};

// Layout of bcd_workspace::small (64-bit words).
constexpr int kSmallWords = 4096;
constexpr int kSmallTable = 0;    // 64 words: slot -> query bits, or per-query scale
constexpr int kSmallOut = 64;     // 64 words: per-slot counts, or per-query sums
constexpr int kSmallBits = 128;   // 64 words: (vertex, bit) pairs to set/clear
constexpr int kSmallBits2 = 192;  // 64 words: (vertex, bit) pairs (query vertices)
constexpr int kSmallSpecs = 256;  // up to 64 draw specs of 6 words

struct bc_graph {
    int32_t n = 0;
    int64_t m = 0;
    bool weighted = false;
    uint32_t max_weight = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int64_t *d_off = nullptr;
    int32_t *d_col = nullptr;
    uint32_t *d_w = nullptr;
    int64_t *d_roff = nullptr;
    int32_t *d_rcol = nullptr;
    uint32_t *d_rw = nullptr;
    std::vector<int64_t> h_off;   // forward offsets (degree checks)
    std::vector<int64_t> h_roff;  // reverse offsets
    std::vector<int32_t> h_hublev; // host copy of the tile ordering key: hop distance to the hub
    std::vector<int64_t> h_twohop; // ... and the arcs two hops away (tie-break)
    int tile_words = 1;           // W of the SPD kernel (unweighted graphs)
    int weighted_words = 1;       // 64-source words of a weighted tile
    int chunk_arcs = 128;
    int source_order = 1;         // 1: tiles ordered by distance to the hub, 0: by vertex id
    int blocks_per_sm = 1;        // resident blocks per SM of the 256-source kernel (1 or 2)
    int block_threads = 512;
    int accumulation = 4;         // 1: Eq. 4 push, 2: vertex scan for one-vertex groups, 3: scan always, 4: chosen per group
    int pull_permille = 0;        // bottom-up levels: frontier out-arcs >= pull_permille / 1000 of m (0: never)
    int wshort = 32;              // weighted kernel: longest row one lane walks alone
    int weighted_kernel = 2;      // weighted graphs: 1 tile kernel, 2 one source per block
    bcd_workspace ws;
    int64_t launches = 0;
    int last_grid = 0;                       // blocks of the last traversal launch
    unsigned long long last_ns_fwd = 0;      // phase times of the last traversal launch
    unsigned long long last_ns_bwd = 0;
    unsigned long long last_ns_other = 0;
    bcd::Counters last;                           // counters of the last traversal launch
    float last_ms_launch = 0;                // CUDA-event time of the last traversal launch
    double timeout_ns = 10.0e9;              // limit on each grid-barrier wait
    std::vector<int32_t> root_cache;         // query vertices whose traversal rlev/rsig or rlevq/rsigq hold
    const void *root_cache_buf = nullptr;    // ... in this buffer (a rebuilt workspace invalidates it)
    int32_t *cancel_h = nullptr;             // pinned, mapped host flag set by bc_cancel
    int32_t *cancel_d = nullptr;             // ... its device address
};

namespace bcd {

// error reporting (thread-local message)
bc_status set_error(bc_status st, const std::string &msg);
bc_status cuda_error(cudaError_t e, const char *what);

#define BCD_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return bcd::cuda_error(e_, #call); \
    } while (0)

#define BCD_TRY(call)                            \
    do {                                         \
        bc_status s_ = (call);                   \
        if (s_ != BC_OK) return s_;              \
    } while (0)

// workspace management (bcd_query.cu)
bc_status ensure_workspace(bc_graph *g, int W);
bc_status grow_history(bc_graph *g);
bc_status alloc_levels(bc_graph *g, int64_t maxlev);
bc_status grow_levels(bc_graph *g);
bc_status grow_buckets(bc_graph *g);
int tile_words_of(const bc_graph *g);  // mask words of the tiles the graph's kernel runs
bc_status ensure_pull_chunks(bc_graph *g);
void free_workspace(bc_graph *g);

// traversal launcher (bcd_traverse.cu)
bc_status run_traversal(bc_graph *g, int W, TravParams &p, int *levels_out, unsigned long long *edges_out);
bc_status launch_weighted(bc_graph *g, TravParams &p);  // bcd_wtraverse.cu
// weighted source kernel (bcd_wsrc.cu): whether a launch goes to it, the
// launcher (same contract as run_traversal) and its state's release
bool src_kernel_applies(const bc_graph *g, const TravParams &p);
bc_status run_src_traversal(bc_graph *g, int W, TravParams &p, int *levels_out, unsigned long long *edges_out);
void free_src_state(bc_graph *g);

// query preparation and slices for the serving loop (bcd_query.cu)
struct PrepItem {
    int32_t r = 0;
    int32_t kind = 0;
    int64_t T = 0;
    uint64_t seed = 0;
    int64_t rv = 0;                 // |RV(r)|
    bool sampled = false;           // resolved: Algorithm 2
    std::vector<int32_t> srcs;      // distinct sources (ascending)
    std::vector<uint32_t> mult;     // draw counts (sampled), parallel to srcs
};
bc_status prepare_sources(bc_graph *g, std::vector<PrepItem> &items);
bc_status set_query_bit(bc_graph *g, int32_t v, int bit, bool on);
bc_status run_slice(bc_graph *g, const std::vector<int32_t> &srcs, const std::vector<uint64_t> &needs,
                    const std::vector<uint32_t> &mult, uint64_t exact_q, const std::vector<int32_t> &slot_roots,
                    std::vector<double> &partials, uint32_t *qflags, unsigned long long *edges);
bc_status check_graph(bc_graph *g, const char *fn);
void begin_call(bc_graph *g);
bc_status prepare_ordering(bc_graph *g);
// Tile order of a source: hop distance to the hub, then arcs two hops away (descending).
int64_t source_order_key(const bc_graph *g, int32_t v);
bc_status ensure_weighted_state(bc_graph *g);
bc_status reset_dense_state(bc_graph *g);

// Host-side fault injection (bc_debug_fail_alloc): true when this
// allocation is the one chosen to fail.
bool inject_alloc_failure();

template <typename T>
bc_status dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (inject_alloc_failure())
        return set_error(BC_E_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                       " bytes failed (injected by bc_debug_fail_alloc)");
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(BC_E_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return BC_OK;
}

template <typename T>
void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace bcd
