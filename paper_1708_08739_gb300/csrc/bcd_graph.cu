// Graph residency: device copy of G, validation (Section 2 graph model) and
// the reverse graph R(G) (Section 4.1, Def. 2), built once per graph.
#include <atomic>
#include <cstring>
#include <string>

#include "bcd_common.cuh"
#include "bcd_scan.cuh"

namespace bcd {

static thread_local std::string t_last_error;

bc_status set_error(bc_status st, const std::string &msg) {
    t_last_error = msg;
    return st;
}

bc_status cuda_error(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return BC_E_OOM;
    return BC_E_CUDA;
}

// Countdown of bc_debug_fail_alloc: the allocation that takes it from 1 to 0
// fails; 0 means off.
static std::atomic<int64_t> g_fail_countdown{0};

bool inject_alloc_failure() {
    int64_t k = g_fail_countdown.load(std::memory_order_relaxed);
    while (k > 0) {
        if (g_fail_countdown.compare_exchange_weak(k, k - 1, std::memory_order_relaxed)) return k == 1;
    }
    return false;
}

namespace {

enum GraphErr : int32_t {
    kGOk = 0,
    kGOffsets = 1,   // offsets not monotone / wrong ends
    kGRange = 2,     // head out of range
    kGLoop = 3,      // self-loop
    kGOrder = 4,     // row not strictly increasing (unsorted or repeated arc)
    kGWeight = 5,    // zero weight
};

__global__ void check_offsets(const int64_t *off, int32_t n, int64_t m, int32_t *err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == 0 && off[0] != 0) atomicMax(err, (int32_t)kGOffsets);
    if (i == n && off[n] != m) atomicMax(err, (int32_t)kGOffsets);
    if (i < n && off[i + 1] < off[i]) atomicMax(err, (int32_t)kGOffsets);
}

// One warp per row: heads in range, no self-loop, strictly increasing.
__global__ void check_rows(const int64_t *off, const int32_t *col, const uint32_t *w, int32_t n, int32_t *err) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (long long u = gw; u < n; u += nw) {
        const long long b = off[u], e = off[u + 1];
        for (long long i = b + lane; i < e; i += 32) {
            const int32_t v = col[i];
            if (v < 0 || v >= n) {
                atomicMax(err, (int32_t)kGRange);
                continue;
            }
            if (v == u) atomicMax(err, (int32_t)kGLoop);
            if (i + 1 < e && col[i + 1] <= v) atomicMax(err, (int32_t)kGOrder);
            if (w && w[i] == 0u) atomicMax(err, (int32_t)kGWeight);
        }
    }
}

__global__ void max_weight(const uint32_t *w, int64_t m, unsigned *out) {
    unsigned mx = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        mx = max(mx, w[i]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void count_heads(const int32_t *col, int64_t m, int64_t *cnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long *)&cnt[col[i]], 1ull);
}

// Scatter of every arc (u, v) of G into row v of R(G) as (v, u).
__global__ void scatter_reverse(const int64_t *off, const int32_t *col, const uint32_t *w, int32_t n,
                                int64_t *cursor, int32_t *rcol, uint32_t *rw) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (long long u = gw; u < n; u += nw) {
        const long long b = off[u], e = off[u + 1];
        for (long long i = b + lane; i < e; i += 32) {
            const int32_t v = col[i];
            const long long pos = (long long)atomicAdd((unsigned long long *)&cursor[v], 1ull);
            rcol[pos] = (int32_t)u;
            if (w) rw[pos] = w[i];
        }
    }
}

}  // namespace

}  // namespace bcd

using namespace bcd;

extern "C" {

const char *bc_last_error(void) { return bcd::t_last_error.c_str(); }

const char *bc_version(void) { return "bcd-gb300 0.1 (sm_103a)"; }

void bc_graph_destroy(bc_graph *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    free_workspace(g);
    if (g->cancel_h) cudaFreeHost(g->cancel_h);
    g->cancel_h = nullptr;
    g->cancel_d = nullptr;
    dev_free(g->d_off);
    dev_free(g->d_col);
    dev_free(g->d_w);
    dev_free(g->d_roff);
    dev_free(g->d_rcol);
    dev_free(g->d_rw);
    delete g;
}

bc_status bc_set_stream(bc_graph *g, void *stream) {
    if (!g) return set_error(BC_E_INVALID_ARG, "bc_set_stream: NULL graph");
    g->stream = (cudaStream_t)stream;
    return BC_OK;
}

bc_status bc_set_config(bc_graph *g, const bc_config *c) {
    if (!g || !c) return set_error(BC_E_INVALID_ARG, "bc_set_config: NULL argument");
    if (c->tile_words && c->tile_words != 1 && c->tile_words != 2 && c->tile_words != 4 && c->tile_words != 8)
        return set_error(BC_E_INVALID_ARG, "bc_set_config: tile_words must be 1, 2, 4 or 8");
    if (c->chunk_arcs && (c->chunk_arcs < 32 || c->chunk_arcs > 65536 || c->chunk_arcs % 32))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: chunk_arcs must be a multiple of 32 in [32, 65536]");
    if (c->block_threads && (c->block_threads < 128 || c->block_threads > 512 || c->block_threads % 32))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: block_threads must be a multiple of 32 in [128, 512]");
    if (c->source_order && c->source_order != 1 && c->source_order != 2)
        return set_error(BC_E_INVALID_ARG, "bc_set_config: source_order must be 1 or 2");
    if (c->source_order) g->source_order = c->source_order == 1 ? 1 : 0;
    if (c->blocks_per_sm && (c->blocks_per_sm < 1 || c->blocks_per_sm > 3))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: blocks_per_sm must be 1, 2 or 3");
    if (c->blocks_per_sm) g->blocks_per_sm = c->blocks_per_sm;
    if (c->weighted_words) {
        const int w = c->weighted_words;
        if (w < 1 || w > 16 || (w & (w - 1)) || (((uint64_t)g->n) << 6) * (uint64_t)w > (1ull << 32))
            return set_error(BC_E_INVALID_ARG, "bc_set_config: weighted_words must be 1, 2, 4, 8 or 16 with n * 64 * weighted_words <= 2^32");
        g->weighted_words = w;
    }
    {
        // the unweighted kernel seeds a tile's S = 64 * tile_words sources with one thread each
        const int tw = c->tile_words ? c->tile_words : g->tile_words;
        const int bt = c->block_threads ? c->block_threads : g->block_threads;
        if (!g->weighted && bt < 64 * tw)
            return set_error(BC_E_INVALID_ARG, "bc_set_config: block_threads must be at least 64 * tile_words");
    }
    if (c->accumulation && (c->accumulation < 1 || c->accumulation > 4))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: accumulation must be 1, 2, 3 or 4");
    if (c->timeout_us < 0) return set_error(BC_E_INVALID_ARG, "bc_set_config: timeout_us must be positive (0 keeps it)");
    if (c->pull_permille && (c->pull_permille < -1 || c->pull_permille > 1000))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: pull_permille must be 1..1000 or -1 (0 keeps it)");
    if (c->pull_permille) g->pull_permille = c->pull_permille < 0 ? 0 : c->pull_permille;
    if (c->weighted_short_row && (c->weighted_short_row < 1 || c->weighted_short_row > 1024))
        return set_error(BC_E_INVALID_ARG, "bc_set_config: weighted_short_row must be 1..1024 (0 keeps it)");
    if (c->weighted_short_row) g->wshort = c->weighted_short_row;
    if (c->weighted_kernel && c->weighted_kernel != 1 && c->weighted_kernel != 2)
        return set_error(BC_E_INVALID_ARG, "bc_set_config: weighted_kernel must be 1 or 2 (0 keeps it)");
    if (c->weighted_kernel) g->weighted_kernel = c->weighted_kernel;
    if (c->timeout_us) g->timeout_ns = 1000.0 * (double)c->timeout_us;
    if (c->accumulation) g->accumulation = c->accumulation;
    if (c->tile_words) g->tile_words = c->tile_words;
    if (c->chunk_arcs) g->chunk_arcs = c->chunk_arcs;
    if (c->block_threads) g->block_threads = c->block_threads;
    return BC_OK;
}

bc_status bc_get_config(const bc_graph *g, bc_config *c) {
    if (!g || !c) return set_error(BC_E_INVALID_ARG, "bc_get_config: NULL argument");
    c->tile_words = g->tile_words;
    c->chunk_arcs = g->chunk_arcs;
    c->block_threads = g->block_threads;
    c->source_order = g->source_order == 1 ? 1 : 2;
    c->blocks_per_sm = g->blocks_per_sm;
    c->weighted_words = g->weighted_words;
    c->accumulation = g->accumulation;
    c->timeout_us = (int32_t)(g->timeout_ns / 1000.0);
    c->pull_permille = g->pull_permille > 0 ? g->pull_permille : -1;
    c->weighted_short_row = g->wshort;
    c->weighted_kernel = g->weighted_kernel;
    return BC_OK;
}

bc_status bc_cancel(bc_graph *g) {
    if (!g) return set_error(BC_E_INVALID_ARG, "bc_cancel: NULL graph");
    if (!g->cancel_h) return set_error(BC_E_INTERNAL, "bc_cancel: the graph has no cancel flag");
    __atomic_store_n(g->cancel_h, 1, __ATOMIC_SEQ_CST);
    return BC_OK;
}

bc_status bc_debug_fail_alloc(int64_t k) {
    if (k < 0) return set_error(BC_E_INVALID_ARG, "bc_debug_fail_alloc: k must be >= 0");
    g_fail_countdown.store(k, std::memory_order_relaxed);
    return BC_OK;
}

bc_status bc_graph_info(const bc_graph *g, int32_t *n, int64_t *m, int32_t *weighted) {
    if (!g) return set_error(BC_E_INVALID_ARG, "bc_graph_info: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (weighted) *weighted = g->weighted ? 1 : 0;
    return BC_OK;
}

bc_status bc_graph_create(const bc_graph_desc *d, bc_graph **out) {
    if (!d || !out) return set_error(BC_E_INVALID_ARG, "bc_graph_create: NULL argument");
    if (d->n <= 0) return set_error(BC_E_INVALID_ARG, "bc_graph_create: n must be positive");
    if (d->m < 0) return set_error(BC_E_INVALID_ARG, "bc_graph_create: m must be non-negative");
    if (!d->row_offsets || (d->m > 0 && !d->cols))
        return set_error(BC_E_INVALID_ARG, "bc_graph_create: NULL offsets or columns");
    if (d->mem_kind != BC_MEM_HOST && d->mem_kind != BC_MEM_DEVICE)
        return set_error(BC_E_INVALID_ARG, "bc_graph_create: mem_kind must be BC_MEM_HOST or BC_MEM_DEVICE");
    bc_graph *g = new bc_graph();
    g->n = d->n;
    g->m = d->m;
    g->weighted = d->weights != nullptr;
    g->stream = (cudaStream_t)d->stream;
    bc_status st = BC_OK;
    auto fail = [&](bc_status s) {
        bc_graph_destroy(g);
        return s;
    };
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "cudaGetDevice"));
    ce = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "cudaDeviceGetAttribute"));
    // the cancel request of bc_cancel: a pinned host word the kernels read
    // through its mapped device address
    if ((ce = cudaHostAlloc((void **)&g->cancel_h, sizeof(int32_t), cudaHostAllocMapped)) != cudaSuccess) {
        g->cancel_h = nullptr;
        return fail(cuda_error(ce, "cudaHostAlloc of the cancel flag"));
    }
    *g->cancel_h = 0;
    if ((ce = cudaHostGetDevicePointer((void **)&g->cancel_d, g->cancel_h, 0)) != cudaSuccess)
        return fail(cuda_error(ce, "cudaHostGetDevicePointer of the cancel flag"));
    const size_t n1 = (size_t)d->n + 1, m = (size_t)d->m;
    if ((st = dev_alloc(&g->d_off, n1)) || (st = dev_alloc(&g->d_col, m)) || (st = dev_alloc(&g->d_roff, n1)) ||
        (st = dev_alloc(&g->d_rcol, m)))
        return fail(st);
    if (g->weighted && ((st = dev_alloc(&g->d_w, m)) || (st = dev_alloc(&g->d_rw, m)))) return fail(st);
    const cudaMemcpyKind kind = d->mem_kind == BC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaStream_t s = g->stream;
    if ((ce = cudaMemcpyAsync(g->d_off, d->row_offsets, n1 * sizeof(int64_t), kind, s)) != cudaSuccess)
        return fail(cuda_error(ce, "copy offsets"));
    if (m && (ce = cudaMemcpyAsync(g->d_col, d->cols, m * sizeof(int32_t), kind, s)) != cudaSuccess)
        return fail(cuda_error(ce, "copy columns"));
    if (g->weighted && m && (ce = cudaMemcpyAsync(g->d_w, d->weights, m * sizeof(uint32_t), kind, s)) != cudaSuccess)
        return fail(cuda_error(ce, "copy weights"));

    // validation
    int32_t *d_err = nullptr;
    if ((st = dev_alloc(&d_err, 1))) return fail(st);
    cudaMemsetAsync(d_err, 0, sizeof(int32_t), s);
    const int tb = 256;
    check_offsets<<<(unsigned)((n1 + tb - 1) / tb), tb, 0, s>>>(g->d_off, d->n, d->m, d_err);
    int32_t herr = 0;
    cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) {
        dev_free(d_err);
        return fail(cuda_error(ce, "validate offsets"));
    }
    if (herr) {
        dev_free(d_err);
        return fail(set_error(BC_E_INVALID_ARG, "bc_graph_create: row offsets must start at 0, end at m and never decrease"));
    }
    const unsigned gblocks = (unsigned)std::max(1, g->num_sms * 8);
    check_rows<<<gblocks, tb, 0, s>>>(g->d_off, g->d_col, g->d_w, d->n, d_err);
    cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) {
        dev_free(d_err);
        return fail(cuda_error(ce, "validate rows"));
    }
    dev_free(d_err);
    switch (herr) {
        case kGOk: break;
        case kGRange: return fail(set_error(BC_E_INVALID_ARG, "bc_graph_create: a column id is outside [0, n)"));
        case kGLoop: return fail(set_error(BC_E_INVALID_GRAPH, "bc_graph_create: self-loop (the graph must be loop-free)"));
        case kGOrder:
            return fail(set_error(BC_E_INVALID_GRAPH,
                                  "bc_graph_create: a row is not strictly increasing (rows must be sorted, without repeated arcs)"));
        case kGWeight: return fail(set_error(BC_E_INVALID_GRAPH, "bc_graph_create: zero weight (weights must be positive)"));
        default: return fail(set_error(BC_E_INTERNAL, "bc_graph_create: unknown validation code"));
    }

    if (g->weighted && m) {
        unsigned *d_mx = nullptr;
        if ((st = dev_alloc(&d_mx, 1))) return fail(st);
        cudaMemsetAsync(d_mx, 0, sizeof(unsigned), s);
        max_weight<<<gblocks, tb, 0, s>>>(g->d_w, d->m, d_mx);
        unsigned hmx = 0;
        cudaMemcpyAsync(&hmx, d_mx, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        ce = cudaStreamSynchronize(s);
        dev_free(d_mx);
        if (ce != cudaSuccess) return fail(cuda_error(ce, "max weight"));
        if (hmx > 4095)
            return fail(set_error(BC_E_INVALID_GRAPH, "bc_graph_create: weights must be at most 4095 (the distance "
                                                      "ring of the weighted kernels has 4096 slots)"));
        g->max_weight = hmx;
    }

    // R(G): in-degree count, exclusive scan, scatter
    int64_t *cnt = nullptr;
    if ((st = dev_alloc(&cnt, n1))) return fail(st);
    cudaMemsetAsync(cnt, 0, n1 * sizeof(int64_t), s);
    if (m) count_heads<<<gblocks, tb, 0, s>>>(g->d_col, d->m, cnt);
    if ((st = scan_exclusive_i64(cnt, g->d_roff, (int64_t)d->n, s)) != BC_OK) {
        dev_free(cnt);
        return fail(st);
    }
    cudaMemcpyAsync(cnt, g->d_roff, (size_t)d->n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (m) scatter_reverse<<<gblocks, tb, 0, s>>>(g->d_off, g->d_col, g->d_w, d->n, cnt, g->d_rcol, g->d_rw);
    g->h_off.resize(n1);
    g->h_roff.resize(n1);
    cudaMemcpyAsync(g->h_off.data(), g->d_off, n1 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(g->h_roff.data(), g->d_roff, n1 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    ce = cudaStreamSynchronize(s);
    dev_free(cnt);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "build reverse graph"));
    if ((ce = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(ce, "graph kernels"));
    g->launches += 5;
    if (!g->weighted) {
        // widest unweighted tile (up to 256 sources) whose per-pair state
        // (sigma and accumulator slabs, 16 bytes per (vertex, source) pair)
        // fits in half of the free device memory; 4-word tiles run two blocks
        // per SM
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        int w = 4;
        while (w > 1 && (double)d->n * 64.0 * w * 16.0 > 0.5 * (double)fr) w >>= 1;
        g->tile_words = w;
        g->blocks_per_sm = 2;
    }
    if (g->weighted) {
        // weighted tile of up to 256 sources (wider tiles measured no faster:
        // sources rarely share a distance, so the work per level grows with
        // the tile), narrower when its per-pair state (dist, sigma, history,
        // bucket share: about 40 bytes) does not fit in half of the free device
        // memory; vertex << log2(S) must fit in 32 bits
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        int nw = 4;
        while (nw > 1 && ((((uint64_t)d->n) << 6) * (uint64_t)nw > (1ull << 32) ||
                          (double)d->n * 64.0 * nw * 40.0 > 0.5 * (double)fr))
            nw >>= 1;
        g->weighted_words = nw;
    }
    *out = g;
    return BC_OK;
}

bc_status bc_graph_reverse(const bc_graph *g, int64_t *roff, int32_t *rcol, uint32_t *rw) {
    if (!g || !roff || (g->m > 0 && !rcol)) return set_error(BC_E_INVALID_ARG, "bc_graph_reverse: NULL argument");
    BCD_CUDA(cudaMemcpyAsync(roff, g->d_roff, ((size_t)g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
    if (g->m)
        BCD_CUDA(cudaMemcpyAsync(rcol, g->d_rcol, (size_t)g->m * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    if (rw && g->weighted && g->m)
        BCD_CUDA(cudaMemcpyAsync(rw, g->d_rw, (size_t)g->m * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
    BCD_CUDA(cudaStreamSynchronize(g->stream));
    return BC_OK;
}

}  // extern "C"
