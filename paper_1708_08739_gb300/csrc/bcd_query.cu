// Query preparation and the public query calls:
//   RV(r) for up to 64 roots at once (reach traversal of R(G), Section 4.1),
//   source sets (Algorithm 1: all of RV(r); Algorithm 2: T Philox draws),
//   the union of source sets of a group (set version, Section 4.2) cut into
//   tiles of S = 64 W sources, the batched SPD/dependency traversal, and the
//   per-query sums (Eq. 5, and Algorithm 2's |RV|/T scaling).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bcd_common.cuh"
#include "bcd_wcols.cuh"
#include "bcd_scan.cuh"

namespace bcd {

namespace {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds; each multiplies words 0 and 2 by the
// round multipliers, mixes the high halves with words 1, 3 and the key, and
// bumps the key by the Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t philox_x0(uint64_t ctr0, uint64_t key0) {
    const uint64_t kMul0 = 0xD2E7470EE14C6C93ull, kMul1 = 0xCA5A826395121157ull;
    const uint64_t kInc0 = 0x9E3779B97F4A7C15ull, kInc1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr0, x1 = 0, x2 = 0, x3 = 0;
    uint64_t k0 = key0, k1 = 0;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hi_a = __umul64hi(kMul0, x0), lo_a = kMul0 * x0;
        const uint64_t hi_b = __umul64hi(kMul1, x2), lo_b = kMul1 * x2;
        const uint64_t y0 = hi_b ^ x1 ^ k0;
        const uint64_t y2 = hi_a ^ x3 ^ k1;
        x0 = y0;
        x1 = lo_b;
        x2 = y2;
        x3 = lo_a;
        k0 += kInc0;
        k1 += kInc1;
    }
    return x0;
}

// Draw t of query q: index floor(x0 * k / 2^64) into the ascending RV list.
struct DrawSpec {
    int64_t first;     // offset of this query's draws in the draw buffer
    int64_t T;
    int64_t list_off;  // offset of its RV list
    int64_t k;         // |RV|
    uint64_t seed;
    int32_t bit;       // query bit in the group
    int32_t pad;
};

static_assert(sizeof(DrawSpec) == 48, "draw spec layout");
static_assert(kSmallSpecs + 64 * sizeof(DrawSpec) / 8 <= kSmallWords, "draw specs fit the staging buffer");

__global__ void draw_kernel(const DrawSpec *specs, int nspec, const int32_t *lists, int32_t *draws,
                            uint64_t *need) {
    const DrawSpec sp = specs[blockIdx.y];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < sp.T;
         t += (long long)gridDim.x * blockDim.x) {
        const uint64_t x0 = philox_x0((uint64_t)t, sp.seed);
        const uint64_t idx = __umul64hi(x0, (uint64_t)sp.k);
        const int32_t v = lists[sp.list_off + (long long)idx];
        draws[sp.first + t] = v;
        if (need) atomicOr((unsigned long long *)&need[v], 1ull << sp.bit);
    }
}

__global__ void mult_kernel(const DrawSpec *specs, const int32_t *draws, const int32_t *posd, uint32_t *mult) {
    const DrawSpec sp = specs[blockIdx.y];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < sp.T;
         t += (long long)gridDim.x * blockDim.x) {
        const int32_t v = draws[sp.first + t];
        atomicAdd(&mult[(size_t)posd[v] * 64 + sp.bit], 1u);
    }
}

// need[v] = OR over slots sl in rvmask[v] of tbl[sl] (exact queries of slot sl)
__global__ void need_from_rv(const uint64_t *rvmask, int64_t n, const uint64_t *tbl, uint64_t *need) {
    __shared__ uint64_t s_tbl[64];
    if (threadIdx.x < 64) s_tbl[threadIdx.x] = tbl[threadIdx.x];
    __syncthreads();
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        uint64_t x = rvmask[v], o = 0;
        while (x) {
            const int b = __ffsll((long long)x) - 1;
            x &= x - 1;
            o |= s_tbl[b];
        }
        need[v] = o;
    }
}

// per-bit population counts of masks[0..n) into cnt[64]
__global__ void bit_counts(const uint64_t *m, int64_t n, unsigned long long *cnt) {
    __shared__ unsigned long long s_cnt[64];
    if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        uint64_t x = m[v];
        while (x) {
            const int b = __ffsll((long long)x) - 1;
            x &= x - 1;
            atomicAdd(&s_cnt[b], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < 64 && s_cnt[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

// set (or clear) one bit at a list of vertices
struct VBit {
    int32_t v;
    int32_t bit;
};

__global__ void set_bits(uint64_t *m, const VBit *list, int cnt, int clear) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const unsigned long long b = 1ull << list[i].bit;
    if (clear)
        atomicAnd((unsigned long long *)&m[list[i].v], ~b);
    else
        atomicOr((unsigned long long *)&m[list[i].v], b);
}

__global__ void fill_i32(int32_t *p, int64_t cnt, int32_t val) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
        p[i] = val;
}

__global__ void positions(const int32_t *list, int64_t cnt, int32_t *pos) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
        pos[list[i]] = (int32_t)i;
}

// bc for each query bit: scale[q] * sum over tiles (pairwise, fixed order)
__global__ void reduce_tiles(const double *tile_partial, int64_t ntiles, const double *scale, double *out) {
    __shared__ double s[256];
    const int q = blockIdx.x;
    double acc = 0.0;
    // each thread a contiguous run of tiles, then a fixed tree
    const long long per = (ntiles + blockDim.x - 1) / blockDim.x;
    const long long t0 = (long long)threadIdx.x * per;
    const long long t1 = (ntiles < t0 + per) ? ntiles : t0 + per;
    for (long long t = t0; t < t1; ++t) acc += tile_partial[t * 64 + q];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = s[0] * scale[q];
}

}  // namespace

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

// Level history and chunk lists. Unweighted entries carry a W-word source
// mask; weighted entries carry one source slot, and the backward partial sums
// of their long rows are indexed by chunk (pcap = ccap). On a
// weighted graph the masks serve only the one-word reach traversals (RV and
// the tile order), which get their own, smaller capacity hmcap.
static bc_status alloc_history(bc_graph *g, int64_t hcap, int64_t ccap, int64_t pcap, int64_t hmcap) {
    bcd_workspace &ws = g->ws;
    dev_free(ws.hv);
    dev_free(ws.hm);
    dev_free(ws.hs);
    dev_free(ws.chunks);
    dev_free(ws.ichunks);
    dev_free(ws.partial);
    dev_free(ws.pdone);
    if (hcap >= (int64_t)INT32_MAX) hcap = (int64_t)INT32_MAX - 1;
    const bool wg = g->weighted;
    if (wg) pcap = ccap;
    hmcap = wg ? std::min(hmcap, hcap) : hcap;
    ws.hmcap = hmcap;
    ws.hcap = hcap;
    ws.ccap = ccap;
    ws.pcap = pcap;
    BCD_TRY(dev_alloc(&ws.hv, (size_t)hcap));
    BCD_TRY(dev_alloc(&ws.hm, wg ? (size_t)hmcap : (size_t)hcap * ws.W));
    BCD_TRY(dev_alloc(&ws.hs, wg ? (size_t)hcap : (size_t)1));
    BCD_TRY(dev_alloc(&ws.chunks, (size_t)ccap));
    BCD_TRY(dev_alloc(&ws.ichunks, wg ? (size_t)1 : (size_t)ccap));
    BCD_TRY(dev_alloc(&ws.partial, wg ? (size_t)pcap : (size_t)1));
    BCD_TRY(dev_alloc(&ws.pdone, wg ? (size_t)pcap : (size_t)1));
    BCD_CUDA(cudaMemsetAsync(ws.pdone, 0, sizeof(int32_t) * (size_t)(wg ? pcap : 1), g->stream));
    return BC_OK;
}

// Per-level arrays of the traversal (entries, chunks, hand-out counters,
// starts; distances for weighted graphs), sized for maxlev levels.
bc_status alloc_levels(bc_graph *g, int64_t maxlev) {
    bcd_workspace &ws = g->ws;
    dev_free(ws.lev_cnt);
    dev_free(ws.lev_ccnt);
    dev_free(ws.lev_grab);
    dev_free(ws.lev_start);
    dev_free(ws.lev_cstart);
    dev_free(ws.lev_icstart);
    dev_free(ws.lev_dist);
    ws.maxlev = (int32_t)maxlev;
    const size_t L = (size_t)maxlev + 2;
    BCD_TRY(dev_alloc(&ws.lev_cnt, L));
    BCD_TRY(dev_alloc(&ws.lev_ccnt, L));
    BCD_TRY(dev_alloc(&ws.lev_grab, 6 * L));
    BCD_TRY(dev_alloc(&ws.lev_start, L));
    BCD_TRY(dev_alloc(&ws.lev_cstart, L));
    BCD_TRY(dev_alloc(&ws.lev_icstart, L));
    if (g->weighted) BCD_TRY(dev_alloc(&ws.lev_dist, L));
    BCD_CUDA(cudaMemsetAsync(ws.lev_cnt, 0, sizeof(unsigned long long) * L, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.lev_ccnt, 0, sizeof(unsigned long long) * L, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.lev_grab, 0, sizeof(unsigned long long) * 6 * L, g->stream));
    return BC_OK;
}

bc_status grow_levels(bc_graph *g) {
    const int64_t cur = g->ws.maxlev;
    if (cur >= (int64_t)INT32_MAX / 4) return set_error(BC_E_OOM, "traversal: more levels than the level arrays can hold");
    const bc_status st = alloc_levels(g, std::min<int64_t>(cur * 4, (int64_t)INT32_MAX / 4));
    if (st != BC_OK) free_workspace(g);
    return st;
}

// Distance slab and bucket ring of the weighted tile kernel. A tile settles each
// (vertex, source) pair once, so the history holds up to n * S entries.
static bc_status build_weighted_state(bc_graph *g);

bc_status ensure_weighted_state(bc_graph *g) {
    if (g->ws.dist) return BC_OK;
    const bc_status st = build_weighted_state(g);
    if (st != BC_OK) free_workspace(g);
    return st;
}

static bc_status build_weighted_state(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    int R = 32;
    while ((uint32_t)R <= g->max_weight) R *= 2;
    if (R > 4096) return set_error(BC_E_INVALID_ARG, "weighted graphs need arc weights of at most 4095");
    ws.ring = R;
    const size_t n = (size_t)g->n;
    const size_t S = 64 * (size_t)ws.W;
    // pending pairs of one distance: a few times the average pairs per
    // distance value (the pairs of a tile spread over hundreds of distances,
    // stale entries included); grown on overflow
    int64_t bcap = 1 << 14;
    while ((size_t)bcap * 64 < n * S) bcap *= 2;
    ws.bcap = bcap;
    BCD_TRY(dev_alloc(&ws.dist, n * S));
    BCD_TRY(dev_alloc(&ws.buckets, (size_t)R * (size_t)bcap));
    BCD_TRY(dev_alloc(&ws.bcount, 2 * (size_t)R));
    BCD_CUDA(cudaMemsetAsync(ws.dist, 0xff, sizeof(uint64_t) * n * S, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.bcount, 0, sizeof(unsigned long long) * 2 * (size_t)R, g->stream));
    const int64_t hneed = std::min<int64_t>((int64_t)(n * S) + 4096, (int64_t)INT32_MAX - 1);
    if (ws.hcap < hneed) BCD_TRY(alloc_history(g, hneed, ws.ccap, ws.pcap, ws.hmcap));
    return BC_OK;
}

// Doubles the entries per slot of the bucket ring (pending pairs of one
// distance outgrew it).
bc_status grow_buckets(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    if (ws.bcap >= ((int64_t)1 << 34)) return set_error(BC_E_OOM, "bucket ring: too many pending pairs at one distance");
    dev_free(ws.buckets);
    ws.bcap *= 2;
    const bc_status st = dev_alloc(&ws.buckets, (size_t)ws.ring * (size_t)ws.bcap);
    if (st != BC_OK) {
        free_workspace(g);
        return st;
    }
    BCD_CUDA(cudaMemsetAsync(ws.bcount, 0, sizeof(unsigned long long) * 2 * (size_t)ws.ring, g->stream));
    return BC_OK;
}

bc_status grow_history(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    if (ws.hcap >= (int64_t)INT32_MAX - 1 && ws.hmcap >= ws.hcap && ws.ccap >= ((int64_t)1 << 34))
        return set_error(BC_E_OOM, "level history exceeds 2^31 entries");
    const bc_status st = alloc_history(g, std::min<int64_t>(ws.hcap * 2, (int64_t)INT32_MAX - 1), ws.ccap * 2,
                                       ws.pcap * 2, ws.hmcap * 2);
    if (st != BC_OK) free_workspace(g);
    return st;
}

int tile_words_of(const bc_graph *g) { return g->weighted ? g->weighted_words : g->tile_words; }

// The in-arcs (R(G)) of every vertex with in-degree > 0, cut into chunks of
// chunk_arcs arcs, as (vertex, chunk index) pairs: the work list of the
// bottom-up forward levels. Built once per graph and chunk size.
bc_status ensure_pull_chunks(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    const int CH = g->chunk_arcs;
    if (ws.pchunks && ws.pchunk_arcs == CH) return BC_OK;
    dev_free(ws.pchunks);
    ws.npchunks = 0;
    std::vector<int2> list;
    list.reserve((size_t)g->n + (size_t)(g->m / CH) + 1);
    for (int32_t v = 0; v < g->n; ++v) {
        const int64_t d = g->h_roff[v + 1] - g->h_roff[v];
        for (int64_t k = 0; k * CH < d; ++k) list.push_back(make_int2(v, (int)k));
    }
    const bc_status st = dev_alloc(&ws.pchunks, std::max<size_t>(list.size(), 1));
    if (st != BC_OK) {
        free_workspace(g);
        return st;
    }
    if (!list.empty())
        BCD_CUDA(cudaMemcpy(ws.pchunks, list.data(), sizeof(int2) * list.size(), cudaMemcpyHostToDevice));
    ws.npchunks = (int64_t)list.size();
    ws.pchunk_arcs = CH;
    return BC_OK;
}

void free_workspace(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    g->root_cache.clear();  // the traversal tables go with the workspace
    g->root_cache_buf = nullptr;
    dev_free(ws.vs);
    dev_free(ws.tag);
    dev_free(ws.sigma);
    dev_free(ws.acc);
    dev_free(ws.hv);
    dev_free(ws.hm);
    dev_free(ws.hs);
    dev_free(ws.chunks);
    dev_free(ws.ichunks);
    dev_free(ws.partial);
    dev_free(ws.pdone);
    dev_free(ws.lev_cnt);
    dev_free(ws.lev_ccnt);
    dev_free(ws.lev_grab);
    dev_free(ws.lev_start);
    dev_free(ws.lev_cstart);
    dev_free(ws.lev_icstart);
    dev_free(ws.pchunks);
    dev_free(ws.rvmask);
    dev_free(ws.need);
    dev_free(ws.qmask);
    dev_free(ws.posd);
    dev_free(ws.hublev);
    dev_free(ws.dist);
    dev_free(ws.buckets);
    dev_free(ws.bcount);
    dev_free(ws.lev_dist);
    dev_free(ws.dlist);
    dev_free(ws.qlevel);
    dev_free(ws.dep);
    dev_free(ws.rlev);
    dev_free(ws.rdist);
    dev_free(ws.rsig);
    dev_free(ws.vsum);
    dev_free(ws.rlevq);
    dev_free(ws.rdistq);
    dev_free(ws.rsigq);
    dev_free(ws.msum);
    dev_free(ws.rtile);
    dev_free(ws.qflags);
    dev_free(ws.srcflag);
    dev_free(ws.ctr);
    dev_free(ws.scratch64);
    dev_free(ws.small);
    dev_free(ws.tile_partial);
    free_src_state(g);
    dev_free(ws.mult);
    dev_free(ws.rvlists);
    dev_free(ws.draws);
    dev_free(ws.blocksums);
    if (ws.pinned) cudaFreeHost(ws.pinned);
    ws = bcd_workspace();
}

static bc_status build_workspace(bc_graph *g, int W);

// The working memory of a handle, allocated on first use. Any failure frees
// all of it (no call can then meet a half-built workspace); the next call
// allocates it again.
bc_status ensure_workspace(bc_graph *g, int W) {
    bcd_workspace &ws = g->ws;
    if (ws.W >= W && ws.vs) return BC_OK;
    const bc_status st = build_workspace(g, W);
    if (st != BC_OK) free_workspace(g);
    return st;
}

static bc_status build_workspace(bc_graph *g, int W) {
    bcd_workspace &ws = g->ws;
    free_workspace(g);
    const int64_t n = g->n, m = g->m;
    ws.W = W;
    ws.n = n;
    ws.m = m;
    // the weighted kernel keeps no masks; the one-word reach traversals do
    ws.vs_stride = g->weighted ? 4 : ((3 * W + 3) / 4) * 4;
    BCD_TRY(dev_alloc(&ws.vs, (size_t)n * ws.vs_stride));
    BCD_TRY(dev_alloc(&ws.tag, (size_t)n));
    BCD_TRY(dev_alloc(&ws.sigma, (size_t)n * 64 * W));
    BCD_TRY(dev_alloc(&ws.acc, g->weighted ? (size_t)1 : (size_t)n * 64 * W));
    const int64_t ch = g->chunk_arcs;
    BCD_TRY(alloc_history(g, 8 * n + 4096, 8 * n + 8 * (m / ch) + 4096, 8 * (m / ch) + 4096, 16 * n + 4096));
    BCD_TRY(alloc_levels(g, std::min<int64_t>(g->weighted ? std::max<int64_t>(n + 1, 65536) : n + 1,
                                              (int64_t)INT32_MAX / 4)));
    BCD_TRY(dev_alloc(&ws.rvmask, (size_t)n));
    BCD_TRY(dev_alloc(&ws.need, (size_t)n));
    BCD_TRY(dev_alloc(&ws.qmask, (size_t)n));
    BCD_TRY(dev_alloc(&ws.posd, (size_t)n));
    BCD_TRY(dev_alloc(&ws.hublev, (size_t)n));
    ws.hub = -1;
    BCD_TRY(dev_alloc(&ws.dlist, (size_t)n + 64 * (size_t)W + 256));  // union padded to whole tiles
    BCD_TRY(dev_alloc(&ws.qlevel, (size_t)64 * W * 64));
    BCD_TRY(dev_alloc(&ws.dep, (size_t)64 * W * 64));
    // vertex scan state
    if (g->weighted)
        BCD_TRY(dev_alloc(&ws.rdist, (size_t)n));
    else
        BCD_TRY(dev_alloc(&ws.rlev, (size_t)n));
    BCD_TRY(dev_alloc(&ws.rsig, (size_t)n));
    BCD_TRY(dev_alloc(&ws.vsum, (size_t)2 * 64 * W));
    BCD_TRY(dev_alloc(&ws.msum, (size_t)2 * 64 * W * 64));
    BCD_TRY(dev_alloc(&ws.rtile, (size_t)64 * W));
    BCD_TRY(dev_alloc(&ws.qflags, 64));
    BCD_TRY(dev_alloc(&ws.srcflag, (size_t)std::max(W, 4)));
    BCD_TRY(dev_alloc(&ws.ctr, 1));
    ws.scratch_len = scan_scratch_len(n) + 64;
    BCD_TRY(dev_alloc(&ws.scratch64, (size_t)ws.scratch_len + 256));
    BCD_TRY(dev_alloc(&ws.small, (size_t)kSmallWords));
    BCD_TRY(reset_dense_state(g));
    BCD_CUDA(cudaMemsetAsync(ws.rvmask, 0, sizeof(uint64_t) * (size_t)n, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.need, 0, sizeof(uint64_t) * (size_t)n, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.qmask, 0, sizeof(uint64_t) * (size_t)n, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.dep, 0, sizeof(double) * 64 * W * 64, g->stream));
    BCD_CUDA(cudaMallocHost(&ws.pinned, 1 << 20));
    ws.pinned_cap = 1 << 20;
    return BC_OK;
}

template <typename T>
static bc_status ensure_buf(T **p, int64_t *cap, int64_t need) {
    if (*cap >= need && *p) return BC_OK;
    dev_free(*p);
    *cap = 0;
    int64_t c = std::max<int64_t>(need, 1024);
    c = c + c / 4;
    BCD_TRY(dev_alloc(p, (size_t)c));
    *cap = c;
    return BC_OK;
}

// ---------------------------------------------------------------------------
// group processing
// ---------------------------------------------------------------------------

struct GQuery {
    int64_t idx;     // index in the caller's array
    int32_t r;
    int32_t kind;    // bc_query_kind after validation
    int64_t T;       // samples (APPROX*, HYBRID tau)
    uint64_t seed;
    int slot;        // RV slot (distinct root)
    bool sampled;    // resolved: Algorithm 2
    int64_t rv;      // |RV(r)|
};

struct GroupTimes {
    float rv = 0, sample = 0, spd = 0, total = 0;
    double fwd = 0, bwd = 0, trav = 0, root = 0;
    bcd::Counters c{};
    int64_t sources = 0;
    int64_t tiles = 0;
    int64_t scan_tiles = 0;  // tiles whose dependencies came from the vertex scan
    unsigned long long eq4_reached = 0, eq4_tight = 0;  // reached / tight pairs of the Eq. 4 tiles
    unsigned long long edges = 0;
    int levels = 0;
};

struct Events {
    cudaEvent_t e[5];
    bool ok = false;
    explicit Events(cudaStream_t s) : stream(s) {
        ok = true;
        for (auto &x : e)
            if (cudaEventCreate(&x) != cudaSuccess) ok = false;
    }
    ~Events() {
        for (auto &x : e) cudaEventDestroy(x);
    }
    void rec(int i) {
        if (ok) cudaEventRecord(e[i], stream);
    }
    float ms(int a, int b) {
        float t = 0;
        if (ok && cudaEventElapsedTime(&t, e[a], e[b]) == cudaSuccess) return t;
        return 0;
    }
    cudaStream_t stream;
};

static unsigned grid_for(const bc_graph *g, int64_t work, int threads) {
    const int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)g->num_sms * 16));
}

// RV for up to 64 distinct roots: rvmask[v] bit sl <=> v in RV(roots[sl]).
bc_status reach_roots(bc_graph *g, const std::vector<int32_t> &roots, std::vector<int64_t> &sizes) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int nr = (int)roots.size();
    BCD_CUDA(cudaMemsetAsync(ws.rvmask, 0, sizeof(uint64_t) * (size_t)g->n, s));
    std::vector<int32_t> tsrc(64, -1);
    for (int i = 0; i < nr; ++i) tsrc[i] = roots[i];
    int32_t *d_tsrc = ws.dlist;  // reused: the union list is built later
    BCD_CUDA(cudaMemcpyAsync(d_tsrc, tsrc.data(), 64 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TravParams p;
    memset(&p, 0, sizeof(p));
    p.mode = kModeReach;
    p.flags = 0;
    p.off = g->d_roff;
    p.col = g->d_rcol;
    p.srcs = d_tsrc;
    p.ntiles = 1;
    p.rvmask = ws.rvmask;
    BCD_TRY(run_traversal(g, 1, p, nullptr, nullptr));
    // r itself is not in RV(r)
    std::vector<VBit> clr(nr);
    for (int i = 0; i < nr; ++i) clr[i] = VBit{roots[i], i};
    VBit *d_clr = (VBit *)(ws.small + kSmallBits);
    BCD_CUDA(cudaMemcpyAsync(d_clr, clr.data(), sizeof(VBit) * nr, cudaMemcpyHostToDevice, s));
    set_bits<<<1, 64, 0, s>>>(ws.rvmask, d_clr, nr, 1);
    unsigned long long *d_cnt = (unsigned long long *)(ws.small + kSmallOut);
    BCD_CUDA(cudaMemsetAsync(d_cnt, 0, 64 * sizeof(unsigned long long), s));
    bit_counts<<<grid_for(g, g->n, 256), 256, 0, s>>>(ws.rvmask, g->n, d_cnt);
    unsigned long long hc[64];
    BCD_CUDA(cudaMemcpyAsync(hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
    BCD_CUDA(cudaStreamSynchronize(s));
    BCD_CUDA(cudaGetLastError());
    g->launches += 3;
    sizes.assign(nr, 0);
    for (int i = 0; i < nr; ++i) sizes[i] = (int64_t)hc[i];
    return BC_OK;
}

// Ascending RV lists of the given slots into ws.rvlists; offsets returned.
bc_status build_rv_lists(bc_graph *g, const std::vector<int> &slots, const std::vector<int64_t> &sizes,
                                std::vector<int64_t> &offs) {
    bcd_workspace &ws = g->ws;
    int64_t total = 0;
    offs.assign(64, -1);
    for (int sl : slots) {
        if (offs[sl] >= 0) continue;
        offs[sl] = total;
        total += sizes[sl];
    }
    BCD_TRY(ensure_buf(&ws.rvlists, &ws.rvlists_cap, total + 1));
    int64_t *d_cnt = ws.scratch64 + ws.scratch_len;  // 1 spare entry past the scan scratch
    for (int sl = 0; sl < 64; ++sl) {
        if (offs[sl] < 0) continue;
        BCD_TRY(compact_mask(ws.rvmask, sl, g->n, ws.rvlists + offs[sl], nullptr, d_cnt, g->stream, ws.scratch64,
                             ws.scratch_len));
        g->launches += 3;
    }
    return BC_OK;
}

// Sum over a vertex's out-arcs of the heads' out-degrees: the arcs two hops
// away, a proxy of how much of the graph a BFS from the vertex reaches by its
// second level.
// One warp per vertex (lanes over its arcs), so hub rows do not hold a thread.
__global__ void two_hop_kernel(const int64_t *off, const int32_t *col, int32_t n, int64_t *out) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        int64_t t = 0;
        for (int64_t a = off[v] + lane; a < off[v + 1]; a += 32) {
            const int32_t w = col[a];
            t += off[w + 1] - off[w];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) out[v] = t;
    }
}

// Tile ordering keys, cached per graph: hop distance from each vertex to the
// hub, the vertex of largest in-degree x out-degree (one reach traversal of
// R(G) from the hub), and the two-hop arc count. Sources at equal distance to
// the hub have closely aligned BFS level profiles, so a tile of them touches
// each vertex at fewer distinct levels; among them, sources of similar
// two-hop reach reach the bulk of the graph at the same level (see
// source_order_key).
static bc_status ensure_hub_levels(bc_graph *g) {
    std::vector<int32_t> &h_lev = g->h_hublev;
    bcd_workspace &ws = g->ws;
    if (ws.hub >= 0 && (int64_t)h_lev.size() == g->n) return BC_OK;
    int32_t hub = 0;
    long long best = -1;
    for (int32_t v = 0; v < g->n; ++v) {
        const long long prod = (long long)(g->h_off[v + 1] - g->h_off[v]) * (g->h_roff[v + 1] - g->h_roff[v]);
        if (prod > best) {
            best = prod;
            hub = v;
        }
    }
    cudaStream_t s = g->stream;
    BCD_CUDA(cudaMemsetAsync(ws.hublev, 0xff, sizeof(int32_t) * (size_t)g->n, s));
    BCD_CUDA(cudaMemsetAsync(ws.rvmask, 0, sizeof(uint64_t) * (size_t)g->n, s));
    std::vector<int32_t> tsrc(64, -1);
    tsrc[0] = hub;
    BCD_CUDA(cudaMemcpyAsync(ws.dlist, tsrc.data(), 64 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TravParams p;
    memset(&p, 0, sizeof(p));
    p.mode = kModeReach;
    p.off = g->d_roff;
    p.col = g->d_rcol;
    p.srcs = ws.dlist;
    p.ntiles = 1;
    p.rvmask = ws.rvmask;
    p.levout = ws.hublev;
    BCD_TRY(run_traversal(g, 1, p, nullptr, nullptr));
    h_lev.resize((size_t)g->n);
    BCD_CUDA(cudaMemcpyAsync(h_lev.data(), ws.hublev, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
    int64_t *d_two = nullptr;
    BCD_TRY(dev_alloc(&d_two, (size_t)g->n));
    two_hop_kernel<<<grid_for(g, (int64_t)g->n * 32, 256), 256, 0, s>>>(g->d_off, g->d_col, g->n, d_two);
    g->launches += 1;
    g->h_twohop.resize((size_t)g->n);
    cudaError_t ce = cudaMemcpyAsync(g->h_twohop.data(), d_two, sizeof(int64_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    dev_free(d_two);
    if (ce != cudaSuccess) return cuda_error(ce, "two-hop counts");
    ws.hub = hub;
    return BC_OK;
}

// Reorder of the source union by source_order_key (ties keep ascending ids).
static bc_status order_sources(bc_graph *g, int64_t nd) {
    bcd_workspace &ws = g->ws;
    BCD_TRY(ensure_hub_levels(g));
    cudaStream_t s = g->stream;
    std::vector<int32_t> d((size_t)nd), out((size_t)nd);
    BCD_CUDA(cudaMemcpyAsync(d.data(), ws.dlist, sizeof(int32_t) * (size_t)nd, cudaMemcpyDeviceToHost, s));
    BCD_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<int64_t, int32_t>> kv((size_t)nd);
    for (int64_t i = 0; i < nd; ++i) kv[i] = {source_order_key(g, d[i]), d[i]};
    std::sort(kv.begin(), kv.end());
    for (int64_t i = 0; i < nd; ++i) out[i] = kv[i].second;
    BCD_CUDA(cudaMemcpyAsync(ws.dlist, out.data(), sizeof(int32_t) * (size_t)nd, cudaMemcpyHostToDevice, s));
    positions<<<grid_for(g, nd, 256), 256, 0, s>>>(ws.dlist, nd, ws.posd);
    g->launches += 1;
    BCD_CUDA(cudaStreamSynchronize(s));
    return BC_OK;
}

static double samples_for(double eps, double delta) { return std::ceil(std::log(2.0 / delta) / (2.0 * eps * eps)); }

// d(r, t) and sigma_rt for every vertex t (the forward pass of Section 2 from
// r alone), kept in rlev / rsig for the vertex scan: a scan-mode launch over
// one tile whose only source is r. Its tile sums are not used (no query takes
// slot 0: exact_q is 0 and there are no draw counts).
static bc_status root_traversal(bc_graph *g, int32_t r) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int W = tile_words_of(g);
    const int S = 64 * W;
    fill_i32<<<1, 256, 0, s>>>(ws.rtile, S, -1);
    fill_i32<<<1, 32, 0, s>>>(ws.rtile, 1, r);
    g->launches += 2;
    if (g->weighted)
        BCD_CUDA(cudaMemsetAsync(ws.rdist, 0xff, sizeof(uint64_t) * (size_t)g->n, s));
    else
        BCD_CUDA(cudaMemsetAsync(ws.rlev, 0xff, sizeof(int32_t) * (size_t)g->n, s));
    BCD_TRY(ensure_buf(&ws.tile_partial, &ws.tile_partial_cap, 64));
    TravParams p;
    memset(&p, 0, sizeof(p));
    p.mode = kModeScan;
    p.flags = kFlagRootOut;
    p.off = g->d_off;
    p.col = g->d_col;
    p.srcs = ws.rtile;
    p.ntiles = 1;
    p.qmask = ws.qmask;
    p.need = ws.need;
    p.exact_q = 0;
    p.mult = nullptr;
    p.qlevel = ws.qlevel;
    p.dep = ws.dep;
    p.tile_partial = ws.tile_partial;
    p.qflags = ws.qflags;
    p.srcflag = ws.srcflag;
    p.rlev = ws.rlev;
    p.rdist = ws.rdist;
    p.rsig = ws.rsig;
    p.vsum = ws.vsum;
    p.vroot = r;
    return run_traversal(g, W, p, nullptr, nullptr);
}

// The vertex scan replaces the Eq. 4 backward for groups whose queries sit at
// one vertex (accumulation 2, the default) or, on unweighted graphs, at up to
// 64 vertices (accumulation 3).
static bool use_vertex_scan(const bc_graph *g, size_t nroots) {
    if (nroots == 1) return g->accumulation >= 2;
    return g->accumulation >= 3 && nroots <= 64;
}

// Cost of one term of the vertex scan (a division and a shared-memory add,
// with the lanes of a warp on one pair's sources) in units of one tight
// (source, arc) pair of the Eq. 4 push (an fp64 reduction). Measured on the
// R-MAT benchmark graphs: 13-20.
constexpr unsigned long long kScanPairCost = 16;

// Offsets in bcd_workspace::small of the column tables of a multi-vertex scan.
constexpr int kSmallQcol = 1024;   // 64 int32: column of each query bit
constexpr int kSmallCroot = 1056;  // 64 int32: vertex of each column
static_assert(kSmallSpecs + 64 * 6 <= kSmallQcol && kSmallCroot + 32 <= kSmallWords, "small table layout");

// d(r_c, t) and sigma_{r_c t} for every vertex t and each of several query
// vertices r_c (the columns): one scan-mode launch over a tile whose slot c
// holds r_c, kept in rlevq / rsigq [t * 64 + c] (unweighted) or rdistq /
// rsigq [t * wcols_stride(K) + c] (weighted).
static bc_status root_traversal_multi(bc_graph *g, const std::vector<int32_t> &roots) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int W = tile_words_of(g);
    const int S = 64 * W;
    const int K = (int)roots.size();
    if (!ws.rsigq) {
        if (g->weighted)
            BCD_TRY(dev_alloc(&ws.rdistq, (size_t)g->n * 64));
        else
            BCD_TRY(dev_alloc(&ws.rlevq, (size_t)g->n * 64));
        bc_status st = dev_alloc(&ws.rsigq, (size_t)g->n * 64);
        if (st != BC_OK) {
            dev_free(ws.rlevq);
            dev_free(ws.rdistq);
            return st;
        }
    }
    if (g->weighted)
        BCD_CUDA(cudaMemsetAsync(ws.rdistq, 0xff, sizeof(uint64_t) * (size_t)g->n * wcols_stride(K), s));
    else
        BCD_CUDA(cudaMemsetAsync(ws.rlevq, 0xff, sizeof(int32_t) * (size_t)g->n * 64, s));
    std::vector<int32_t> tsrc(S, -1);
    for (int c = 0; c < K; ++c) tsrc[c] = roots[c];
    BCD_CUDA(cudaMemcpyAsync(ws.rtile, tsrc.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    BCD_TRY(ensure_buf(&ws.tile_partial, &ws.tile_partial_cap, 64));
    TravParams p;
    memset(&p, 0, sizeof(p));
    p.mode = kModeScan;
    p.flags = kFlagRootOut;
    p.off = g->d_off;
    p.col = g->d_col;
    p.srcs = ws.rtile;
    p.ntiles = 1;
    p.qmask = ws.qmask;
    p.need = ws.need;
    p.exact_q = 0;
    p.mult = nullptr;
    p.qlevel = ws.qlevel;
    p.dep = ws.dep;
    p.tile_partial = ws.tile_partial;
    p.qflags = ws.qflags;
    p.srcflag = ws.srcflag;
    p.rlev = ws.rlev;
    p.rsig = ws.rsig;
    p.vsum = ws.vsum;
    p.ncols = K;
    p.qcol = (const int32_t *)(ws.small + kSmallQcol);  // uploaded by the caller
    p.croot = (const int32_t *)(ws.small + kSmallCroot);
    p.rlevq = ws.rlevq;
    p.rdistq = ws.rdistq;
    p.rsigq = ws.rsigq;
    p.msum = ws.msum;
    p.vroot = roots[0];
    return run_traversal(g, W, p, nullptr, nullptr);
}

// Tiles [lo, hi) of shard k out of nshards contiguous shards of ntiles tiles.
static void shard_tiles(int64_t ntiles, int32_t k, int32_t nshards, int64_t *lo, int64_t *hi) {
    *lo = ntiles * k / nshards;
    *hi = ntiles * (k + 1) / nshards;
}

// Runs one group of at most 64 queries whose out-degree is positive; with
// nshards > 1 only the group's tiles of shard k run, and each score is that
// shard's part of the sum (already scaled by |RV| / T for sampled queries).
// The traversal from the query vertices that the vertex scan reads: from one
// vertex (rlev, rsig) or from several columns (rlevq, rsigq, with the column
// tables qcol / croot staged in the small buffer). Kept across calls while the
// ordered list of vertices is unchanged (it depends on the graph only).
static bc_status scan_roots(bc_graph *g, const std::vector<int32_t> &roots, const std::vector<int32_t> &qcol,
                            double *ms_root) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    if (roots.size() >= 2) {
        std::vector<int32_t> croot(64, 0);
        for (size_t c = 0; c < roots.size(); ++c) croot[c] = roots[c];
        BCD_CUDA(cudaMemcpyAsync(ws.small + kSmallQcol, qcol.data(), 64 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        BCD_CUDA(cudaMemcpyAsync(ws.small + kSmallCroot, croot.data(), 64 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (g->root_cache == roots && ws.rsigq && g->root_cache_buf == (const void *)ws.rsigq) return BC_OK;
        g->root_cache.clear();
        BCD_TRY(root_traversal_multi(g, roots));
        g->root_cache = roots;
        g->root_cache_buf = ws.rsigq;
    } else {
        const void *buf = g->weighted ? (const void *)ws.rdist : (const void *)ws.rlev;
        if (g->root_cache == roots && g->root_cache_buf == buf) return BC_OK;
        g->root_cache.clear();
        BCD_TRY(root_traversal(g, roots[0]));
        g->root_cache = roots;
        g->root_cache_buf = buf;
    }
    *ms_root += g->last_ms_launch;
    return BC_OK;
}

static bc_status run_group(bc_graph *g, std::vector<GQuery> &qs, bc_result *res, GroupTimes &tm, int32_t shard,
                           int32_t nshards) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int nq = (int)qs.size();
    const int W = tile_words_of(g);
    const int S = 64 * W;
    // the ordering key's reach traversal uses the union buffer: run it first
    if (g->source_order == 1) BCD_TRY(ensure_hub_levels(g));
    Events ev(s);
    ev.rec(0);
    // distinct roots
    std::vector<int32_t> roots;
    for (auto &q : qs) {
        auto it = std::find(roots.begin(), roots.end(), q.r);
        if (it == roots.end()) {
            q.slot = (int)roots.size();
            roots.push_back(q.r);
        } else {
            q.slot = (int)(it - roots.begin());
        }
    }
    std::vector<int64_t> sizes;
    BCD_TRY(reach_roots(g, roots, sizes));
    ev.rec(1);
    // resolve kinds, need bits of exact queries
    uint64_t exact_q = 0;
    std::vector<uint64_t> tbl(64, 0);
    std::vector<int> sampled_slots;
    for (int i = 0; i < nq; ++i) {
        GQuery &q = qs[i];
        q.rv = sizes[q.slot];
        q.sampled = (q.kind == BC_QUERY_APPROX || q.kind == BC_QUERY_APPROX_T ||
                     (q.kind == BC_QUERY_HYBRID && q.rv > q.T));
        if (q.sampled && q.rv > 0) {
            sampled_slots.push_back(q.slot);
        } else if (!q.sampled) {
            exact_q |= 1ull << i;
            tbl[q.slot] |= 1ull << i;
        }
    }
    uint64_t *d_tbl = ws.small + kSmallTable;
    BCD_CUDA(cudaMemcpyAsync(d_tbl, tbl.data(), 64 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    need_from_rv<<<grid_for(g, g->n, 256), 256, 0, s>>>(ws.rvmask, g->n, d_tbl, ws.need);
    g->launches += 1;
    // sampled queries: RV lists and draws
    std::vector<DrawSpec> specs;
    int64_t total_draws = 0;
    if (!sampled_slots.empty()) {
        std::vector<int64_t> offs;
        BCD_TRY(build_rv_lists(g, sampled_slots, sizes, offs));
        for (int i = 0; i < nq; ++i) {
            GQuery &q = qs[i];
            if (!q.sampled || q.rv == 0) continue;
            DrawSpec d;
            d.first = total_draws;
            d.T = q.T;
            d.list_off = offs[q.slot];
            d.k = q.rv;
            d.seed = q.seed;
            d.bit = i;
            d.pad = 0;
            specs.push_back(d);
            total_draws += q.T;
        }
        BCD_TRY(ensure_buf(&ws.draws, &ws.draws_cap, total_draws + 1));
        DrawSpec *d_specs = (DrawSpec *)(ws.small + kSmallSpecs);
        BCD_CUDA(cudaMemcpyAsync(d_specs, specs.data(), sizeof(DrawSpec) * specs.size(), cudaMemcpyHostToDevice, s));
        int64_t maxT = 0;
        for (auto &d : specs) maxT = std::max(maxT, d.T);
        dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((maxT + 255) / 256, 4096)), (unsigned)specs.size());
        draw_kernel<<<grid, 256, 0, s>>>(d_specs, (int)specs.size(), ws.rvlists, ws.draws, ws.need);
        g->launches += 1;
    }
    // union of the source sets, padded to whole tiles
    int64_t *d_cnt = ws.scratch64 + ws.scratch_len;
    BCD_TRY(compact_mask(ws.need, -1, g->n, ws.dlist, ws.posd, d_cnt, s, ws.scratch64, ws.scratch_len));
    g->launches += 3;
    int64_t nd = 0;
    BCD_CUDA(cudaMemcpyAsync(&nd, d_cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BCD_CUDA(cudaStreamSynchronize(s));
    const int64_t ntiles = (nd + S - 1) / S;
    int64_t t_lo = 0, t_hi = ntiles;
    shard_tiles(ntiles, shard, nshards, &t_lo, &t_hi);
    const int64_t nrun = t_hi - t_lo;  // tiles this call runs
    if (g->source_order == 1 && ntiles >= 2) BCD_TRY(order_sources(g, nd));
    if (ntiles * S > nd) {
        fill_i32<<<1, 256, 0, s>>>(ws.dlist + nd, ntiles * S - nd, -1);
        g->launches += 1;
    }
    if (!specs.empty()) {
        BCD_TRY(ensure_buf(&ws.mult, &ws.mult_cap, std::max<int64_t>(ntiles, 1) * S * 64));
        BCD_CUDA(cudaMemsetAsync(ws.mult, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles, 1) * S * 64, s));
        DrawSpec *d_specs = (DrawSpec *)(ws.small + kSmallSpecs);
        BCD_CUDA(cudaMemcpyAsync(d_specs, specs.data(), sizeof(DrawSpec) * specs.size(), cudaMemcpyHostToDevice, s));
        int64_t maxT = 0;
        for (auto &d : specs) maxT = std::max(maxT, d.T);
        dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((maxT + 255) / 256, 4096)), (unsigned)specs.size());
        mult_kernel<<<grid, 256, 0, s>>>(d_specs, ws.draws, ws.posd, ws.mult);
        g->launches += 1;
    }
    // query vertices
    std::vector<VBit> qb(nq);
    for (int i = 0; i < nq; ++i) qb[i] = VBit{qs[i].r, i};
    VBit *d_qb = (VBit *)(ws.small + kSmallBits2);
    BCD_CUDA(cudaMemcpyAsync(d_qb, qb.data(), sizeof(VBit) * nq, cudaMemcpyHostToDevice, s));
    set_bits<<<1, 64, 0, s>>>(ws.qmask, d_qb, nq, 0);
    g->launches += 1;
    // the query bits must leave qmask on every exit (an error included), or a
    // later group would read them as its own; a failed allocation may have
    // freed the workspace, and qmask with it
    struct QmaskGuard {
        bc_graph *g;
        std::vector<VBit> bits;
        bool armed = true;
        ~QmaskGuard() {
            if (!armed || !g->ws.qmask || !g->ws.small) return;
            VBit *d = (VBit *)(g->ws.small + kSmallBits2);
            if (cudaMemcpyAsync(d, bits.data(), sizeof(VBit) * bits.size(), cudaMemcpyHostToDevice, g->stream) ==
                cudaSuccess) {
                set_bits<<<1, 64, 0, g->stream>>>(g->ws.qmask, d, (int)bits.size(), 1);
                g->launches += 1;
            }
            cudaStreamSynchronize(g->stream);
            cudaGetLastError();
        }
    } qguard{g, qb};
    BCD_CUDA(cudaMemsetAsync(ws.qflags, 0, 64 * sizeof(uint32_t), s));
    ev.rec(2);
    // batched SPD + dependencies over all tiles
    std::vector<double> sums(64, 0.0);
    std::vector<uint32_t> qflags(64, 0);
    int levels = 0;
    unsigned long long edges = 0;
    const bool scan = nrun > 0 && use_vertex_scan(g, roots.size());
    const bool multi = scan && roots.size() >= 2;
    if (scan) {
        std::vector<int32_t> qcol(64, 0);
        for (int i = 0; i < nq; ++i) qcol[i] = qs[i].slot;
        BCD_TRY(scan_roots(g, roots, qcol, &tm.root));
    }
    if (nrun > 0) {
        BCD_TRY(ensure_buf(&ws.tile_partial, &ws.tile_partial_cap, nrun * 64));
        // tiles [first, first + count) of this call's range, in scan or Eq. 4 mode
        auto launch_tiles = [&](bool scan_mode, int64_t first, int64_t count) -> bc_status {
            TravParams p;
            memset(&p, 0, sizeof(p));
            p.mode = scan_mode ? kModeScan : kModeSpd;
            p.flags = 0;
            if (scan_mode) {
                p.rlev = ws.rlev;
                p.rdist = ws.rdist;
                p.rsig = ws.rsig;
                p.vsum = ws.vsum;
                p.vroot = roots[0];
            }
            if (scan_mode && multi) {
                p.ncols = (int32_t)roots.size();
                p.qcol = (const int32_t *)(ws.small + kSmallQcol);
                p.croot = (const int32_t *)(ws.small + kSmallCroot);
                p.rlevq = ws.rlevq;
                p.rdistq = ws.rdistq;
                p.rsigq = ws.rsigq;
                p.msum = ws.msum;
            }
            p.off = g->d_off;
            p.col = g->d_col;
            p.srcs = ws.dlist + (t_lo + first) * S;
            p.ntiles = count;
            p.qmask = ws.qmask;
            p.need = ws.need;
            p.exact_q = exact_q;
            p.mult = specs.empty() ? nullptr : ws.mult + (size_t)(t_lo + first) * S * 64;
            p.qlevel = ws.qlevel;
            p.dep = ws.dep;
            p.tile_partial = ws.tile_partial + first * 64;
            p.qflags = ws.qflags;
            p.srcflag = ws.srcflag;
            int lv = 0;
            unsigned long long ed = 0;
            BCD_TRY(src_kernel_applies(g, p) ? run_src_traversal(g, W, p, &lv, &ed) : run_traversal(g, W, p, &lv, &ed));
            levels = std::max(levels, lv);
            edges += ed;
            tm.fwd += g->last_ns_fwd * 1e-6;
            tm.bwd += g->last_ns_bwd * 1e-6;
            tm.trav += g->last_ms_launch;
            const Counters &c = g->last;
            tm.c.reached += c.reached;
            tm.c.tight += c.tight;
            tm.c.arc_visits += c.arc_visits;
            tm.c.vb += c.vb;
            tm.c.eb += c.eb;
            tm.c.vpairs += c.vpairs;
            tm.c.pull_levels += c.pull_levels;
            if (!scan_mode) {
                tm.eq4_reached += c.reached;
                tm.eq4_tight += c.tight;
            }
            return BC_OK;
        };
        std::vector<uint32_t> cal_flags(64, 0);
        if (multi && g->accumulation == 4 && nrun > 1) {
            // choose the backward on the group's first tile: the scan's terms
            // (a division and a shared-memory add each) against the push's
            // tight (source, arc) pairs (an fp64 reduction each), at the
            // measured cost ratio of about 16
            BCD_TRY(launch_tiles(true, 0, 1));
            BCD_CUDA(cudaMemcpyAsync(cal_flags.data(), ws.qflags, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            BCD_CUDA(cudaStreamSynchronize(s));
            const bool scan_rest = g->last.vpairs * kScanPairCost <= g->last.tight;
            tm.scan_tiles += 1;
            BCD_TRY(launch_tiles(scan_rest, 1, nrun - 1));
            if (scan_rest) tm.scan_tiles += nrun - 1;
        } else {
            BCD_TRY(launch_tiles(scan, 0, nrun));
            if (scan) tm.scan_tiles += nrun;
        }
        std::vector<double> scale(64, 1.0);
        for (int i = 0; i < nq; ++i)
            if (qs[i].sampled && qs[i].rv > 0) scale[i] = (double)qs[i].rv / (double)qs[i].T;
        double *d_scale = (double *)(ws.small + kSmallTable);
        double *d_out = (double *)(ws.small + kSmallOut);
        BCD_CUDA(cudaMemcpyAsync(d_scale, scale.data(), 64 * sizeof(double), cudaMemcpyHostToDevice, s));
        reduce_tiles<<<64, 256, 0, s>>>(ws.tile_partial, nrun, d_scale, d_out);
        BCD_CUDA(cudaMemcpyAsync(sums.data(), d_out, 64 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BCD_CUDA(cudaMemcpyAsync(qflags.data(), ws.qflags, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BCD_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < 64; ++i) qflags[i] |= cal_flags[i];
        g->launches += 1;
    }
    set_bits<<<1, 64, 0, s>>>(ws.qmask, d_qb, nq, 1);
    g->launches += 1;
    qguard.armed = false;
    ev.rec(3);
    BCD_CUDA(cudaStreamSynchronize(s));
    BCD_CUDA(cudaGetLastError());
    for (int i = 0; i < nq; ++i) {
        bc_result &o = res[qs[i].idx];
        o.status = BC_OK;
        o.bc = sums[i];
        o.flags = (qflags[i] & 1u) ? BC_FLAG_SIGMA_2_53 : 0u;
        o.rv_size = qs[i].rv;
        o.samples = (qs[i].sampled && qs[i].rv > 0) ? qs[i].T : 0;
    }
    tm.rv = ev.ms(0, 1);
    tm.sample = ev.ms(1, 2);
    tm.spd = ev.ms(2, 3);
    tm.total = ev.ms(0, 3);
    tm.sources = nrun == ntiles ? nd : std::max<int64_t>(0, std::min(nd, t_hi * S) - t_lo * S);
    tm.tiles = nrun;
    tm.edges = edges;
    tm.levels = levels;
    return BC_OK;
}

// ---------------------------------------------------------------------------
// helpers for the serving loop (bcd_server.cu)
// ---------------------------------------------------------------------------

bc_status prepare_sources(bc_graph *g, std::vector<PrepItem> &items) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    std::vector<int32_t> roots;
    std::vector<int> slot_of(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        auto it = std::find(roots.begin(), roots.end(), items[i].r);
        slot_of[i] = (int)(it - roots.begin());
        if (it == roots.end()) roots.push_back(items[i].r);
    }
    if (roots.size() > 64) return set_error(BC_E_INTERNAL, "prepare_sources: more than 64 roots");
    std::vector<int64_t> sizes;
    BCD_TRY(reach_roots(g, roots, sizes));
    std::vector<int> slots;
    for (size_t sl = 0; sl < roots.size(); ++sl)
        if (sizes[sl] > 0) slots.push_back((int)sl);
    std::vector<int64_t> offs;
    int64_t total = 0;
    for (int sl : slots) total += sizes[sl];
    std::vector<int32_t> lists((size_t)std::max<int64_t>(total, 1));
    if (!slots.empty()) {
        BCD_TRY(build_rv_lists(g, slots, sizes, offs));
        BCD_CUDA(cudaMemcpyAsync(lists.data(), ws.rvlists, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, s));
    }
    // draws of the sampled items
    std::vector<DrawSpec> specs;
    int64_t ndraws = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        PrepItem &it = items[i];
        it.rv = sizes[slot_of[i]];
        it.sampled = it.kind == BC_QUERY_APPROX || it.kind == BC_QUERY_APPROX_T ||
                     (it.kind == BC_QUERY_HYBRID && it.rv > it.T);
        if (it.sampled && it.rv > 0) {
            DrawSpec d;
            d.first = ndraws;
            d.T = it.T;
            d.list_off = offs[slot_of[i]];
            d.k = it.rv;
            d.seed = it.seed;
            d.bit = 0;
            d.pad = 0;
            specs.push_back(d);
            ndraws += it.T;
        }
    }
    std::vector<int32_t> draws((size_t)std::max<int64_t>(ndraws, 1));
    if (!specs.empty()) {
        BCD_TRY(ensure_buf(&ws.draws, &ws.draws_cap, ndraws + 1));
        // specs go up in groups of 64 (the staging buffer holds 64)
        for (size_t b = 0; b < specs.size(); b += 64) {
            const size_t nb = std::min<size_t>(64, specs.size() - b);
            DrawSpec *d_specs = (DrawSpec *)(ws.small + kSmallSpecs);
            BCD_CUDA(cudaMemcpyAsync(d_specs, specs.data() + b, sizeof(DrawSpec) * nb, cudaMemcpyHostToDevice, s));
            int64_t maxT = 0;
            for (size_t k = b; k < b + nb; ++k) maxT = std::max(maxT, specs[k].T);
            dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((maxT + 255) / 256, 4096)), (unsigned)nb);
            draw_kernel<<<grid, 256, 0, s>>>(d_specs, (int)nb, ws.rvlists, ws.draws, nullptr);
            BCD_CUDA(cudaStreamSynchronize(s));
            g->launches += 1;
        }
        BCD_CUDA(cudaMemcpyAsync(draws.data(), ws.draws, sizeof(int32_t) * (size_t)ndraws, cudaMemcpyDeviceToHost, s));
    }
    BCD_CUDA(cudaStreamSynchronize(s));
    BCD_CUDA(cudaGetLastError());
    size_t si = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        PrepItem &it = items[i];
        it.srcs.clear();
        it.mult.clear();
        if (it.rv == 0) continue;
        if (!it.sampled) {
            const int32_t *b = lists.data() + offs[slot_of[i]];
            it.srcs.assign(b, b + it.rv);
        } else {
            const DrawSpec &d = specs[si++];
            std::vector<int32_t> dv(draws.begin() + d.first, draws.begin() + d.first + d.T);
            std::sort(dv.begin(), dv.end());
            for (size_t k = 0; k < dv.size();) {
                size_t j = k;
                while (j < dv.size() && dv[j] == dv[k]) ++j;
                it.srcs.push_back(dv[k]);
                it.mult.push_back((uint32_t)(j - k));
                k = j;
            }
        }
    }
    return BC_OK;
}

bc_status set_query_bit(bc_graph *g, int32_t v, int bit, bool on) {
    VBit b{v, bit};
    VBit *d = (VBit *)(g->ws.small + kSmallBits2);
    BCD_CUDA(cudaMemcpyAsync(d, &b, sizeof(VBit), cudaMemcpyHostToDevice, g->stream));
    set_bits<<<1, 32, 0, g->stream>>>(g->ws.qmask, d, 1, on ? 0 : 1);
    BCD_CUDA(cudaStreamSynchronize(g->stream));
    g->launches += 1;
    return BC_OK;
}

__global__ void scatter_need(const int32_t *v, const uint64_t *mask, int64_t cnt, uint64_t *need) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
        need[v[i]] = mask[i];
}

bc_status run_slice(bc_graph *g, const std::vector<int32_t> &srcs, const std::vector<uint64_t> &needs,
                    const std::vector<uint32_t> &mult, uint64_t exact_q, const std::vector<int32_t> &slot_roots,
                    std::vector<double> &partials, uint32_t *qflags, unsigned long long *edges) {
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int W = tile_words_of(g);
    const int S = 64 * W;
    const int64_t ntiles = (int64_t)srcs.size() / S;
    if (ntiles * S != (int64_t)srcs.size() || ntiles == 0) return set_error(BC_E_INTERNAL, "run_slice: ragged slice");
    std::vector<int32_t> vs;
    std::vector<uint64_t> ms;
    uint64_t used = 0;  // query slots some source of the slice serves
    for (size_t i = 0; i < srcs.size(); ++i)
        if (srcs[i] >= 0) {
            vs.push_back(srcs[i]);
            ms.push_back(needs[i]);
            used |= needs[i];
        }
    BCD_CUDA(cudaMemcpyAsync(ws.dlist, srcs.data(), sizeof(int32_t) * srcs.size(), cudaMemcpyHostToDevice, s));
    BCD_TRY(ensure_buf(&ws.draws, &ws.draws_cap, (int64_t)vs.size() * 3 + 4));
    int32_t *d_v = ws.draws;
    uint64_t *d_m = (uint64_t *)(ws.draws + ((vs.size() + 3) & ~(size_t)1));
    BCD_CUDA(cudaMemcpyAsync(d_v, vs.data(), sizeof(int32_t) * vs.size(), cudaMemcpyHostToDevice, s));
    BCD_CUDA(cudaMemcpyAsync(d_m, ms.data(), sizeof(uint64_t) * ms.size(), cudaMemcpyHostToDevice, s));
    scatter_need<<<grid_for(g, (int64_t)vs.size(), 256), 256, 0, s>>>(d_v, d_m, (int64_t)vs.size(), ws.need);
    const bool any_mult = !mult.empty();
    if (any_mult) {
        BCD_TRY(ensure_buf(&ws.mult, &ws.mult_cap, (int64_t)mult.size()));
        BCD_CUDA(cudaMemcpyAsync(ws.mult, mult.data(), sizeof(uint32_t) * mult.size(), cudaMemcpyHostToDevice, s));
    }
    BCD_TRY(ensure_buf(&ws.tile_partial, &ws.tile_partial_cap, ntiles * 64));
    BCD_CUDA(cudaMemsetAsync(ws.qflags, 0, 64 * sizeof(uint32_t), s));
    // the query vertices of the slots this slice serves, as scan columns
    std::vector<int32_t> roots, qcol(64, 0);
    for (int q = 0; q < 64; ++q) {
        if (!((used >> q) & 1ull) || q >= (int)slot_roots.size() || slot_roots[q] < 0) continue;
        auto it = std::find(roots.begin(), roots.end(), slot_roots[q]);
        qcol[q] = (int)(it - roots.begin());
        if (it == roots.end()) roots.push_back(slot_roots[q]);
    }
    const bool scan = !roots.empty() && use_vertex_scan(g, roots.size());
    const bool multi = scan && roots.size() >= 2;
    double ms_root = 0.0;
    if (scan) BCD_TRY(scan_roots(g, roots, qcol, &ms_root));
    auto launch = [&](bool scan_mode, int64_t first, int64_t count) -> bc_status {
        TravParams p;
        memset(&p, 0, sizeof(p));
        p.mode = scan_mode ? kModeScan : kModeSpd;
        if (scan_mode) {
            p.rlev = ws.rlev;
            p.rdist = ws.rdist;
            p.rsig = ws.rsig;
            p.vsum = ws.vsum;
            p.vroot = roots[0];
        }
        if (scan_mode && multi) {
            p.ncols = (int32_t)roots.size();
            p.qcol = (const int32_t *)(ws.small + kSmallQcol);
            p.croot = (const int32_t *)(ws.small + kSmallCroot);
            p.rlevq = ws.rlevq;
            p.rdistq = ws.rdistq;
            p.rsigq = ws.rsigq;
            p.msum = ws.msum;
        }
        p.off = g->d_off;
        p.col = g->d_col;
        p.srcs = ws.dlist + first * S;
        p.ntiles = count;
        p.qmask = ws.qmask;
        p.need = ws.need;
        p.exact_q = exact_q;
        p.mult = any_mult ? ws.mult + (size_t)first * S * 64 : nullptr;
        p.qlevel = ws.qlevel;
        p.dep = ws.dep;
        p.tile_partial = ws.tile_partial + first * 64;
        p.qflags = ws.qflags;
        p.srcflag = ws.srcflag;
        g->launches += 1;
        unsigned long long ed = 0;
        BCD_TRY(src_kernel_applies(g, p) ? run_src_traversal(g, W, p, nullptr, &ed)
                                          : run_traversal(g, W, p, nullptr, &ed));
        if (edges) *edges += ed;
        return BC_OK;
    };
    if (edges) *edges = 0;
    std::vector<uint32_t> cal_flags(64, 0);
    if (multi && g->accumulation == 4 && ntiles > 1) {
        BCD_TRY(launch(true, 0, 1));
        BCD_CUDA(cudaMemcpyAsync(cal_flags.data(), ws.qflags, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BCD_CUDA(cudaStreamSynchronize(s));
        BCD_TRY(launch(g->last.vpairs * kScanPairCost <= g->last.tight, 1, ntiles - 1));
    } else {
        BCD_TRY(launch(scan, 0, ntiles));
    }
    partials.resize((size_t)ntiles * 64);
    BCD_CUDA(cudaMemcpyAsync(partials.data(), ws.tile_partial, sizeof(double) * partials.size(), cudaMemcpyDeviceToHost, s));
    BCD_CUDA(cudaMemcpyAsync(qflags, ws.qflags, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCD_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 64; ++i) qflags[i] |= cal_flags[i];
    return BC_OK;
}

int64_t source_order_key(const bc_graph *g, int32_t v) {
    if (g->source_order != 1) return v;
    constexpr int64_t kLow = ((int64_t)1 << 40) - 1;
    int64_t lev = 0, two = 0;
    if ((int64_t)g->h_hublev.size() == g->n) lev = g->h_hublev[v] < 0 ? ((1 << 22) - 1) : std::min(g->h_hublev[v], (1 << 22) - 2);
    if ((int64_t)g->h_twohop.size() == g->n) two = std::min<int64_t>(g->h_twohop[v], kLow);
    return (lev << 40) | (kLow - two);
}

bc_status prepare_ordering(bc_graph *g) { return g->source_order == 1 ? ensure_hub_levels(g) : BC_OK; }

// A call starts: a cancel request left from before it is dropped.
void begin_call(bc_graph *g) {
    if (g->cancel_h) __atomic_store_n(g->cancel_h, 0, __ATOMIC_SEQ_CST);
}

bc_status check_graph(bc_graph *g, const char *fn) {
    if (!g) return set_error(BC_E_INVALID_ARG, std::string(fn) + ": NULL graph");
    begin_call(g);
    BCD_TRY(ensure_workspace(g, tile_words_of(g)));
    if (g->weighted) BCD_TRY(ensure_weighted_state(g));
    return BC_OK;
}

static bc_status run_batch(bc_graph *g, const bc_query *queries, int64_t nq, bc_result *out, bc_batch_info *info,
                           int32_t shard = 0, int32_t nshards = 1) {
    if (!g) return set_error(BC_E_INVALID_ARG, "bc_batch: NULL graph");
    if (nshards < 1 || shard < 0 || shard >= nshards)
        return set_error(BC_E_INVALID_ARG, "bc_batch_shard: need 0 <= shard < nshards");
    if (nq < 0 || (nq > 0 && (!queries || !out))) return set_error(BC_E_INVALID_ARG, "bc_batch: bad query array");
    BCD_TRY(check_graph(g, "bc_batch"));
    const int64_t launches0 = g->launches;
    bc_batch_info bi;
    memset(&bi, 0, sizeof(bi));
    bi.queries = nq;
    std::vector<GQuery> group;
    auto flush = [&]() -> bc_status {
        if (group.empty()) return BC_OK;
        GroupTimes t;
        bc_status st = run_group(g, group, out, t, shard, nshards);
        if (st != BC_OK) {
            for (auto &q : group) out[q.idx].status = st;
            group.clear();
            return st;
        }
        bi.sources_run += t.sources;
        bi.edges_traversed += (int64_t)t.edges;
        bi.ms_rv += t.rv;
        bi.ms_sample += t.sample;
        bi.ms_spd += t.spd;
        bi.ms_total += t.total;
        bi.ms_forward += t.fwd;
        bi.ms_backward += t.bwd;
        bi.tiles += t.tiles;
        bi.max_level = std::max(bi.max_level, (int32_t)t.levels);
        bi.grid_blocks = g->last_grid;
        bi.ms_traversal += t.trav;
        bi.reached_pairs += (int64_t)t.c.reached;
        bi.tight_pairs += (int64_t)t.c.tight;
        bi.arc_visits += (int64_t)t.c.arc_visits;
        bi.union_vertices += (int64_t)t.c.vb;
        bi.union_arcs += (int64_t)t.c.eb;
        bi.scan_pairs += (int64_t)t.c.vpairs;
        bi.pull_levels += (int64_t)t.c.pull_levels;
        bi.scan_tiles += t.scan_tiles;
        bi.eq4_reached_pairs += (int64_t)t.eq4_reached;
        bi.eq4_tight_pairs += (int64_t)t.eq4_tight;
        bi.ms_root += t.root;
        group.clear();
        return BC_OK;
    };
    bc_status worst = BC_OK;
    for (int64_t i = 0; i < nq; ++i) {
        const bc_query &q = queries[i];
        bc_result &o = out[i];
        memset(&o, 0, sizeof(o));
        if (q.r < 0 || q.r >= g->n) {
            o.status = set_error(BC_E_INVALID_ARG, "query vertex out of range");
            continue;
        }
        GQuery gq;
        gq.idx = i;
        gq.r = q.r;
        gq.kind = q.kind;
        gq.seed = q.seed;
        gq.T = 0;
        gq.slot = 0;
        gq.sampled = false;
        gq.rv = 0;
        if (q.kind == BC_QUERY_EXACT) {
        } else if (q.kind == BC_QUERY_APPROX) {
            if (!(q.eps > 0.0) || !(q.delta > 0.0 && q.delta < 1.0)) {
                o.status = set_error(BC_E_INVALID_ARG, "approx query needs eps > 0 and 0 < delta < 1");
                continue;
            }
            const double T = samples_for(q.eps, q.delta);
            if (!(T >= 1.0) || T > 4.0e9) {
                o.status = set_error(BC_E_INVALID_ARG, "approx query: sample count out of range");
                continue;
            }
            gq.T = (int64_t)T;
        } else if (q.kind == BC_QUERY_APPROX_T || q.kind == BC_QUERY_HYBRID) {
            if (q.T < 1 || q.T > 4000000000ll) {
                o.status = set_error(BC_E_INVALID_ARG, "query T must be in [1, 4e9]");
                continue;
            }
            gq.T = q.T;
        } else {
            o.status = set_error(BC_E_INVALID_ARG, "unknown query kind");
            continue;
        }
        // Prop. 1 / Algorithm 1: out-degree 0 => BC(r) = 0 without traversal
        if (g->h_off[q.r + 1] == g->h_off[q.r]) {
            o.status = BC_OK;
            o.bc = 0.0;
            o.flags = BC_FLAG_TRIVIAL_ZERO;
            continue;
        }
        group.push_back(gq);
        if (group.size() == 64) {
            bc_status st = flush();
            if (st != BC_OK) worst = st;
        }
    }
    bc_status st = flush();
    if (st != BC_OK) worst = st;
    bi.launches = g->launches - launches0;
    if (info) *info = bi;
    if (worst == BC_E_CUDA || worst == BC_E_OOM || worst == BC_E_TIMEOUT || worst == BC_E_INTERNAL ||
        worst == BC_E_CANCELLED)
        return worst;
    return BC_OK;
}

}  // namespace bcd

using namespace bcd;

extern "C" {

bc_status bc_samples_for(double eps, double delta, int64_t *T) {
    if (!T) return set_error(BC_E_INVALID_ARG, "bc_samples_for: NULL output");
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0))
        return set_error(BC_E_INVALID_ARG, "bc_samples_for: need eps > 0 and 0 < delta < 1");
    const double t = bcd::samples_for(eps, delta);
    if (!(t >= 1.0) || t > 4.0e9) return set_error(BC_E_INVALID_ARG, "bc_samples_for: sample count out of range");
    *T = (int64_t)t;
    return BC_OK;
}

bc_status bc_batch(bc_graph *g, const bc_query *queries, int64_t nq, bc_result *out, bc_batch_info *info) {
    return run_batch(g, queries, nq, out, info);
}

bc_status bc_batch_shard(bc_graph *g, const bc_query *queries, int64_t nq, int32_t shard, int32_t nshards,
                         bc_result *out, bc_batch_info *info) {
    return run_batch(g, queries, nq, out, info, shard, nshards);
}

static bc_status single(bc_graph *g, const bc_query &q, double *bc, bc_info *info) {
    if (!bc) return set_error(BC_E_INVALID_ARG, "NULL result pointer");
    bc_result r;
    bc_batch_info bi;
    BCD_TRY(run_batch(g, &q, 1, &r, &bi));
    if (r.status != BC_OK) return (bc_status)r.status;
    *bc = r.bc;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->rv_size = r.rv_size;
        info->samples = r.samples;
        info->sources_run = bi.sources_run;
        info->edges_traversed = bi.edges_traversed;
        info->max_level = bi.max_level;
        info->flags = r.flags;
        info->ms_rv = bi.ms_rv;
        info->ms_sample = bi.ms_sample;
        info->ms_spd = bi.ms_spd;
        info->ms_total = bi.ms_total;
    }
    return BC_OK;
}

bc_status bc_exact(bc_graph *g, int32_t r, double *bc, bc_info *info) {
    bc_query q;
    memset(&q, 0, sizeof(q));
    q.r = r;
    q.kind = BC_QUERY_EXACT;
    return single(g, q, bc, info);
}

bc_status bc_approx(bc_graph *g, int32_t r, double eps, double delta, uint64_t seed, double *bc, bc_info *info) {
    bc_query q;
    memset(&q, 0, sizeof(q));
    q.r = r;
    q.kind = BC_QUERY_APPROX;
    q.eps = eps;
    q.delta = delta;
    q.seed = seed;
    return single(g, q, bc, info);
}

bc_status bc_approx_T(bc_graph *g, int32_t r, int64_t T, uint64_t seed, double *bc, bc_info *info) {
    bc_query q;
    memset(&q, 0, sizeof(q));
    q.r = r;
    q.kind = BC_QUERY_APPROX_T;
    q.T = T;
    q.seed = seed;
    return single(g, q, bc, info);
}

bc_status bc_rv_compute(bc_graph *g, int32_t r, int32_t *out, int64_t cap, int64_t *count) {
    if (!g || !count) return set_error(BC_E_INVALID_ARG, "bc_rv_compute: NULL argument");
    if (r < 0 || r >= g->n) return set_error(BC_E_INVALID_ARG, "bc_rv_compute: vertex out of range");
    if (cap < 0 || (cap > 0 && !out)) return set_error(BC_E_INVALID_ARG, "bc_rv_compute: bad output buffer");
    begin_call(g);
    BCD_TRY(ensure_workspace(g, tile_words_of(g)));
    std::vector<int64_t> sizes;
    BCD_TRY(reach_roots(g, std::vector<int32_t>{r}, sizes));
    *count = sizes[0];
    if (cap < sizes[0]) return set_error(BC_E_BUFFER_TOO_SMALL, "bc_rv_compute: output capacity below |RV(r)|");
    std::vector<int64_t> offs;
    BCD_TRY(build_rv_lists(g, std::vector<int>{0}, sizes, offs));
    if (sizes[0] > 0)
        BCD_CUDA(cudaMemcpyAsync(out, g->ws.rvlists, sizeof(int32_t) * (size_t)sizes[0], cudaMemcpyDeviceToHost,
                                 g->stream));
    BCD_CUDA(cudaStreamSynchronize(g->stream));
    return BC_OK;
}

bc_status bc_draw_samples(bc_graph *g, int32_t r, int64_t T, uint64_t seed, int32_t *out, int64_t *rv_size) {
    if (!g || !rv_size) return set_error(BC_E_INVALID_ARG, "bc_draw_samples: NULL argument");
    if (r < 0 || r >= g->n) return set_error(BC_E_INVALID_ARG, "bc_draw_samples: vertex out of range");
    if (T < 1 || T > 4000000000ll || !out) return set_error(BC_E_INVALID_ARG, "bc_draw_samples: bad T or output");
    begin_call(g);
    BCD_TRY(ensure_workspace(g, tile_words_of(g)));
    *rv_size = 0;
    if (g->h_off[r + 1] == g->h_off[r]) return BC_OK;
    std::vector<int64_t> sizes;
    BCD_TRY(reach_roots(g, std::vector<int32_t>{r}, sizes));
    if (sizes[0] == 0) return BC_OK;
    *rv_size = sizes[0];
    std::vector<int64_t> offs;
    BCD_TRY(build_rv_lists(g, std::vector<int>{0}, sizes, offs));
    BCD_TRY(ensure_buf(&g->ws.draws, &g->ws.draws_cap, T + 1));
    DrawSpec d;
    d.first = 0;
    d.T = T;
    d.list_off = 0;
    d.k = sizes[0];
    d.seed = seed;
    d.bit = 0;
    d.pad = 0;
    DrawSpec *d_spec = (DrawSpec *)(g->ws.small + kSmallSpecs);
    BCD_CUDA(cudaMemcpyAsync(d_spec, &d, sizeof(d), cudaMemcpyHostToDevice, g->stream));
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((T + 255) / 256, 4096)), 1);
    draw_kernel<<<grid, 256, 0, g->stream>>>(d_spec, 1, g->ws.rvlists, g->ws.draws, nullptr);
    BCD_CUDA(cudaMemcpyAsync(out, g->ws.draws, sizeof(int32_t) * (size_t)T, cudaMemcpyDeviceToHost, g->stream));
    BCD_CUDA(cudaStreamSynchronize(g->stream));
    BCD_CUDA(cudaGetLastError());
    return BC_OK;
}

// Autotuner: coordinate descent over the launch parameters, each candidate
// timed (CUDA events of the group, second of two runs) on a probe batch made
// of the caller's queries with every query turned into A-BCD with at most
// probe_T draws (same vertices and seeds, so the same mix of query vertices
// and the same shape of source sets, at a small cost per candidate).
bc_status bc_tune(bc_graph *g, const bc_query *queries, int64_t nq, int64_t probe_T, bc_config *best,
                  bc_tune_report *rep) {
    if (!g || !best || (nq > 0 && !queries) || nq < 1) return set_error(BC_E_INVALID_ARG, "bc_tune: bad arguments");
    if (probe_T < 1 || probe_T > 1000000) return set_error(BC_E_INVALID_ARG, "bc_tune: probe_T must be 1..10^6");
    const int64_t n = std::min<int64_t>(nq, 64);
    std::vector<bc_query> probe((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        probe[i] = queries[i];
        int64_t T = probe_T;
        if (queries[i].kind == BC_QUERY_APPROX_T) T = std::min<int64_t>(queries[i].T, probe_T);
        probe[i].kind = BC_QUERY_APPROX_T;
        probe[i].T = T;
    }
    std::vector<bc_result> out((size_t)n);
    bc_config cur;
    BCD_TRY(bc_get_config(g, &cur));
    const bc_config start = cur;
    int runs = 0;
    auto timed = [&](const bc_config &c, double *ms) -> bc_status {
        BCD_TRY(bc_set_config(g, &c));
        bc_batch_info bi;
        BCD_TRY(run_batch(g, probe.data(), n, out.data(), &bi));  // warm (workspace, chunk lists)
        BCD_TRY(run_batch(g, probe.data(), n, out.data(), &bi));
        *ms = bi.ms_total;
        ++runs;
        return BC_OK;
    };
    double best_ms = 0.0;
    BCD_TRY(timed(cur, &best_ms));
    const double start_ms = best_ms;
    // the search space, one parameter at a time (0 ends a list)
    std::vector<std::pair<int32_t bc_config::*, std::vector<int32_t>>> space;
    if (g->weighted) {
        space.push_back({&bc_config::weighted_kernel, {1, 2}});
        space.push_back({&bc_config::weighted_words, {2, 4, 8}});
        space.push_back({&bc_config::weighted_short_row, {16, 32, 64}});
        space.push_back({&bc_config::chunk_arcs, {64, 128, 256}});
        space.push_back({&bc_config::accumulation, {1, 4}});
    } else {
        space.push_back({&bc_config::tile_words, {2, 4, 8}});
        space.push_back({&bc_config::blocks_per_sm, {1, 2}});
        space.push_back({&bc_config::chunk_arcs, {64, 128, 256}});
        space.push_back({&bc_config::pull_permille, {-1, 200}});
        space.push_back({&bc_config::accumulation, {1, 4}});
    }
    for (auto &dim : space) {
        for (int32_t val : dim.second) {
            if (cur.*(dim.first) == val) continue;
            bc_config c = cur;
            c.*(dim.first) = val;
            if (!g->weighted && c.block_threads < 64 * c.tile_words) continue;
            if ((((uint64_t)g->n) << 6) * (uint64_t)c.weighted_words > (1ull << 32)) continue;
            double ms = 0.0;
            bc_status st = timed(c, &ms);
            if (st == BC_E_OOM) {  // a wider tile that does not fit: skip it
                BCD_TRY(bc_set_config(g, &cur));
                continue;
            }
            if (st != BC_OK) {
                bc_set_config(g, &start);
                return st;
            }
            if (ms < best_ms) {
                best_ms = ms;
                cur = c;
            }
        }
    }
    BCD_TRY(bc_set_config(g, &cur));
    *best = cur;
    if (rep) {
        rep->candidates = runs;
        rep->ms_default = start_ms;
        rep->ms_best = best_ms;
        rep->probe_queries = n;
    }
    return BC_OK;
}

bc_status bc_spd_probe(bc_graph *g, const int32_t *sources, int32_t nsrc, const int32_t *targets, int32_t nt,
                       uint64_t *dist, double *sigma, double *dep, uint32_t *flags) {
    if (!g || (nsrc > 0 && !sources) || (nt > 0 && !targets))
        return set_error(BC_E_INVALID_ARG, "bc_spd_probe: NULL argument");
    if (nt < 0 || nt > 64) return set_error(BC_E_INVALID_ARG, "bc_spd_probe: 0..64 targets");
    BCD_TRY(check_graph(g, "bc_spd_probe"));
    bcd_workspace &ws = g->ws;
    cudaStream_t s = g->stream;
    const int W = tile_words_of(g);  // one tile of the graph's kernel; slots past nsrc stay empty
    const int S = 64 * W;
    if (nsrc < 1 || nsrc > S)
        return set_error(BC_E_INVALID_ARG, "bc_spd_probe: 1..64*tile_words sources (one tile of the kernel)");
    for (int i = 0; i < nsrc; ++i) {
        if (sources[i] < 0 || sources[i] >= g->n) return set_error(BC_E_INVALID_ARG, "bc_spd_probe: source out of range");
        for (int j = 0; j < i; ++j)
            if (sources[j] == sources[i]) return set_error(BC_E_INVALID_ARG, "bc_spd_probe: sources must be distinct");
    }
    for (int j = 0; j < nt; ++j)
        if (targets[j] < 0 || targets[j] >= g->n) return set_error(BC_E_INVALID_ARG, "bc_spd_probe: target out of range");
    const uint64_t tbits = nt == 64 ? ~0ull : ((1ull << nt) - 1ull);
    std::vector<int32_t> tsrc(S, -1);
    for (int i = 0; i < nsrc; ++i) tsrc[i] = sources[i];
    BCD_CUDA(cudaMemcpyAsync(ws.dlist, tsrc.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    // need: every source needs every target; qmask: target bits
    std::vector<VBit> nb, qb;
    for (int i = 0; i < nsrc; ++i)
        for (int j = 0; j < nt; ++j) nb.push_back(VBit{sources[i], j});
    for (int j = 0; j < nt; ++j) qb.push_back(VBit{targets[j], j});
    VBit *d_nb = nullptr;
    BCD_TRY(dev_alloc(&d_nb, nb.size() + qb.size() + 1));
    if (!nb.empty() || !qb.empty())
        BCD_CUDA(cudaMemcpyAsync(d_nb, nb.empty() ? qb.data() : nb.data(), sizeof(VBit) * nb.size(),
                                 cudaMemcpyHostToDevice, s));
    if (!qb.empty())
        BCD_CUDA(cudaMemcpyAsync(d_nb + nb.size(), qb.data(), sizeof(VBit) * qb.size(), cudaMemcpyHostToDevice, s));
    BCD_CUDA(cudaMemsetAsync(ws.need, 0, sizeof(uint64_t) * (size_t)g->n, s));
    if (!nb.empty()) set_bits<<<(unsigned)((nb.size() + 255) / 256), 256, 0, s>>>(ws.need, d_nb, (int)nb.size(), 0);
    if (!qb.empty()) set_bits<<<1, 64, 0, s>>>(ws.qmask, d_nb + nb.size(), (int)qb.size(), 0);
    BCD_TRY(ensure_buf(&ws.tile_partial, &ws.tile_partial_cap, 64));
    BCD_CUDA(cudaMemsetAsync(ws.dep, 0, sizeof(double) * S * 64, s));
    BCD_CUDA(cudaMemsetAsync(ws.qflags, 0, 64 * sizeof(uint32_t), s));
    TravParams p;
    memset(&p, 0, sizeof(p));
    p.mode = kModeSpd;
    p.off = g->d_off;
    p.col = g->d_col;
    p.srcs = ws.dlist;
    p.ntiles = 1;
    p.qmask = ws.qmask;
    p.need = ws.need;
    p.exact_q = tbits;
    p.qlevel = ws.qlevel;
    p.dep = ws.dep;
    p.tile_partial = ws.tile_partial;
    p.qflags = ws.qflags;
    p.srcflag = ws.srcflag;
    bc_status st = BC_OK;
    if (dist || sigma || flags) {
        p.flags = kFlagNoBackward | kFlagNoReset;
        st = run_traversal(g, W, p, nullptr, nullptr);
        if (st == BC_OK && g->weighted) {
            // export the first nsrc columns of the dist and sigma slabs [v][S]
            const size_t n = (size_t)g->n;
            std::vector<uint64_t> wd(dist ? n * nsrc : 0);
            std::vector<double> sg(sigma ? n * nsrc : 0);
            std::vector<uint64_t> sf(W);
            if (dist)
                BCD_CUDA(cudaMemcpy2DAsync(wd.data(), sizeof(uint64_t) * nsrc, ws.dist, sizeof(uint64_t) * S,
                                           sizeof(uint64_t) * nsrc, n, cudaMemcpyDeviceToHost, s));
            if (sigma)
                BCD_CUDA(cudaMemcpy2DAsync(sg.data(), sizeof(double) * nsrc, ws.sigma, sizeof(double) * S,
                                           sizeof(double) * nsrc, n, cudaMemcpyDeviceToHost, s));
            BCD_CUDA(cudaMemcpyAsync(sf.data(), ws.srcflag, sizeof(uint64_t) * W, cudaMemcpyDeviceToHost, s));
            cudaError_t ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) st = cuda_error(ce, "probe export");
            if (st == BC_OK) {
                for (int i = 0; i < nsrc; ++i)
                    for (size_t v = 0; v < n; ++v) {
                        if (dist) dist[(size_t)i * n + v] = wd[v * nsrc + i];
                        if (sigma) sigma[(size_t)i * n + v] = sg[v * nsrc + i];
                    }
                if (flags)
                    for (int i = 0; i < nsrc; ++i) flags[i] = ((sf[i >> 6] >> (i & 63)) & 1ull) ? BC_FLAG_SIGMA_2_53 : 0u;
            }
        } else if (st == BC_OK) {
            // export sigma [v][S] and the level history
            const size_t n = (size_t)g->n;
            std::vector<double> sg;
            if (sigma) {
                sg.resize(n * S);
                cudaMemcpyAsync(sg.data(), ws.sigma, sizeof(double) * n * S, cudaMemcpyDeviceToHost, s);
            }
            std::vector<unsigned long long> lc(ws.maxlev + 2);
            cudaMemcpyAsync(lc.data(), ws.lev_cnt, sizeof(unsigned long long) * lc.size(), cudaMemcpyDeviceToHost, s);
            std::vector<uint64_t> sf(W);
            cudaMemcpyAsync(sf.data(), ws.srcflag, sizeof(uint64_t) * W, cudaMemcpyDeviceToHost, s);
            cudaError_t ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) st = cuda_error(ce, "probe export");
            int64_t total = 0;
            const int levels = (int)std::min<unsigned long long>(g->last.levels_max + 1, (unsigned long long)ws.maxlev + 1);
            for (int L = 0; L < levels; ++L) total += (int64_t)lc[L];
            std::vector<int32_t> hv(std::max<int64_t>(total, 1));
            std::vector<uint64_t> hm(std::max<int64_t>(total, 1) * W);
            if (st == BC_OK && total > 0) {
                cudaMemcpyAsync(hv.data(), ws.hv, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(hm.data(), ws.hm, sizeof(uint64_t) * total * W, cudaMemcpyDeviceToHost, s);
                ce = cudaStreamSynchronize(s);
                if (ce != cudaSuccess) st = cuda_error(ce, "probe export");
            }
            if (st == BC_OK) {
                if (dist) std::fill(dist, dist + (size_t)nsrc * n, ~0ull);
                if (sigma) std::fill(sigma, sigma + (size_t)nsrc * n, 0.0);
                int64_t e = 0;
                for (int L = 0; L < levels; ++L) {
                    for (unsigned long long k = 0; k < lc[L]; ++k, ++e) {
                        const int32_t v = hv[e];
                        for (int i = 0; i < nsrc; ++i) {
                            if ((hm[e * W + (i >> 6)] >> (i & 63)) & 1ull) {
                                if (dist) dist[(size_t)i * n + v] = (uint64_t)L;
                                if (sigma) sigma[(size_t)i * n + v] = sg[(size_t)v * S + i];
                            }
                        }
                    }
                }
                if (flags)
                    for (int i = 0; i < nsrc; ++i) flags[i] = ((sf[i >> 6] >> (i & 63)) & 1ull) ? BC_FLAG_SIGMA_2_53 : 0u;
            }
        }
        bc_status st2 = reset_dense_state(g);
        if (st == BC_OK) st = st2;
    }
    if (st == BC_OK && dep) {
        p.flags = 0;
        BCD_CUDA(cudaMemsetAsync(ws.dep, 0, sizeof(double) * S * 64, s));
        st = run_traversal(g, W, p, nullptr, nullptr);
        if (st == BC_OK) {
            std::vector<double> hd((size_t)S * 64);
            BCD_CUDA(cudaMemcpyAsync(hd.data(), ws.dep, sizeof(double) * S * 64, cudaMemcpyDeviceToHost, s));
            BCD_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i < nsrc; ++i)
                for (int j = 0; j < nt; ++j) dep[(size_t)i * nt + j] = hd[i * 64 + j];
        }
    }
    if (!qb.empty() && ws.qmask) set_bits<<<1, 64, 0, s>>>(ws.qmask, d_nb + nb.size(), (int)qb.size(), 1);
    cudaStreamSynchronize(s);
    dev_free(d_nb);
    return st;
}

}  // extern "C"
