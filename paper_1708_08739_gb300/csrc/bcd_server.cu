// Serving loop with continuous batching (set version of Section 4.2 applied
// over time).
//
// A worker thread owns the graph. Submitted queries wait in a queue until a
// query slot (one of 64 mask bits) is free; then their source sets are
// prepared (RV(r) by one reach traversal for up to 64 roots, Philox draws for
// sampled queries). A prepared query is admitted while the device bytes that
// its sources hold, added to those of the queries already admitted, fit the
// server's byte budget; otherwise it goes back to the head of the queue until
// others finish, and a query that alone exceeds the budget is answered with
// BC_E_BUSY. An admitted query's sources join a pool of pending sources: a
// source already pending for an earlier query is shared (the new query's bit
// is added to it). The worker runs the pool in slices of tiles, taking sources
// round-robin across the active queries, so that queries that arrive while
// others are running get their tiles into the very next slice and their work
// overlaps on the device. Each query sums its per-tile partials in slice order
// and completes when its last source has run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bcd_common.cuh"

using Clock = std::chrono::steady_clock;

namespace {

struct SQuery {
    uint64_t ticket = 0;
    bc_query q{};
    int slot = -1;
    bool sampled = false;
    int64_t rv = 0;
    int64_t T = 0;
    int64_t outstanding = 0;
    double acc = 0.0;
    uint32_t flags = 0;
    int32_t status = BC_OK;
    bool done = false;
    std::deque<int32_t> pending;                 // sources not yet run
    std::unordered_map<int32_t, uint32_t> mult;  // draw counts (sampled)
    int64_t bytes = 0;                           // device bytes its sources hold (staged_bytes)
    Clock::time_point t_submit, t_done;
    bc_result res{};
};

double samples_for(double eps, double delta) { return std::ceil(std::log(2.0 / delta) / (2.0 * eps * eps)); }

}  // namespace

// Device bytes that a query's distinct sources hold from admission until they
// have run: per source, its slot in the union list (4 bytes), its query mask
// (8 bytes) and, for a sampled query, its row of draw counts (64 x 4 bytes);
// per tile of S sources, the tile's per-query partial sums (64 x 8 bytes).
// The per-(vertex, source) slabs (sigma, accumulators, masks, level history)
// are allocated once per graph for one tile and reused by every tile, so they
// are the server's fixed cost, outside the budget.
int64_t bcd_staged_bytes(int64_t sources, bool sampled, int S) {
    const int64_t per = 4 + 8 + (sampled ? 64 * 4 : 0);
    return sources * per + (sources + S - 1) / S * 64 * 8;
}

struct bc_server {
    bc_graph *g = nullptr;
    bc_server_config cfg{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<SQuery *> queue;
    std::unordered_map<uint64_t, SQuery *> tickets;
    bc_server_stats stats{};  // guarded by mu
    // worker-owned state
    SQuery *slots[64] = {};
    int nactive = 0;
    int rr = 0;                                       // round-robin cursor over slots
    int64_t held_bytes = 0;                           // sum of the admitted queries' bytes
    int64_t defer_held = -1;                          // held_bytes when the queue head was deferred
    std::unordered_map<int32_t, uint64_t> pend_need;  // pending source -> slots that need it
    bc_status fatal = BC_OK;

    void run();
    bool admit();
    bool run_slice_once();
    void complete(SQuery *q, int32_t status);
    void fail_active(int32_t status);
};

void bc_server::complete(SQuery *q, int32_t status) {
    q->res.status = status;
    q->res.bc = q->acc * (q->sampled && q->rv > 0 ? (double)q->rv / (double)q->T : 1.0);
    q->res.flags = q->flags;
    q->res.rv_size = q->rv;
    q->res.samples = (q->sampled && q->rv > 0) ? q->T : 0;
    q->pending.clear();
    held_bytes -= q->bytes;
    q->bytes = 0;
    if (q->slot >= 0) {
        // a failed allocation may have freed the workspace (and the query
        // masks with it)
        if (g->ws.qmask) bcd::set_query_bit(g, q->q.r, q->slot, false);
        slots[q->slot] = nullptr;
        --nactive;
        q->slot = -1;
    }
    std::lock_guard<std::mutex> lk(mu);
    q->t_done = Clock::now();
    q->done = true;
    stats.completed += 1;
    stats.active = nactive;
    cv_done.notify_all();
}

// Every active query ends with status (a slice failed, or the workspace that
// held their query masks was freed); their pending sources leave the pool.
void bc_server::fail_active(int32_t status) {
    for (int s = 0; s < 64; ++s)
        if (slots[s]) complete(slots[s], status);
    pend_need.clear();
}

// Moves queued queries into free slots, prepares their sources, and merges
// them into the pending pool while their bytes fit the budget. Returns true
// if any query left the queue.
bool bc_server::admit() {
    // a deferred head waits until running queries have freed some bytes
    if (defer_held >= 0 && nactive > 0 && held_bytes >= defer_held) return false;
    defer_held = -1;
    std::vector<SQuery *> batch;
    {
        std::lock_guard<std::mutex> lk(mu);
        while (!queue.empty() && nactive + (int)batch.size() < cfg.max_active && held_bytes < cfg.max_device_bytes) {
            batch.push_back(queue.front());
            queue.pop_front();
        }
    }
    if (batch.empty()) return false;
    std::vector<bcd::PrepItem> items;
    std::vector<SQuery *> prepq;
    for (SQuery *q : batch) {
        // Prop. 1 / Algorithm 1: out-degree 0 => 0 without traversal
        if (g->h_off[q->q.r + 1] == g->h_off[q->q.r]) {
            q->flags = BC_FLAG_TRIVIAL_ZERO;
            complete(q, BC_OK);
            continue;
        }
        bcd::PrepItem it;
        it.r = q->q.r;
        it.kind = q->q.kind;
        it.T = q->T;
        it.seed = q->q.seed;
        items.push_back(it);
        prepq.push_back(q);
    }
    if (items.empty()) return true;
    bc_status st = bcd::prepare_sources(g, items);
    if (st != BC_OK) {
        for (SQuery *q : prepq) complete(q, st);
        if (!g->ws.qmask) fail_active(st);
        return true;
    }
    const int S = 64 * bcd::tile_words_of(g);
    std::vector<SQuery *> deferred;
    for (size_t i = 0; i < prepq.size(); ++i) {
        SQuery *q = prepq[i];
        bcd::PrepItem &it = items[i];
        q->rv = it.rv;
        q->sampled = it.sampled;
        if (it.srcs.empty()) {
            complete(q, BC_OK);
            continue;
        }
        const int64_t bytes = bcd_staged_bytes((int64_t)it.srcs.size(), q->sampled, S);
        if (bytes > cfg.max_device_bytes) {
            // could never fit, even alone
            bcd::set_error(BC_E_BUSY, "bc_server: the query's sources need more device bytes than the budget");
            complete(q, BC_E_BUSY);
            continue;
        }
        if (held_bytes + bytes > cfg.max_device_bytes) {
            deferred.push_back(q);  // waits for running queries to free their bytes
            continue;
        }
        int slot = 0;
        while (slots[slot]) ++slot;
        slots[slot] = q;
        q->slot = slot;
        ++nactive;
        q->bytes = bytes;
        held_bytes += bytes;
        if (bcd::set_query_bit(g, q->q.r, slot, true) != BC_OK) {
            complete(q, BC_E_CUDA);
            continue;
        }
        const uint64_t bit = 1ull << slot;
        for (size_t k = 0; k < it.srcs.size(); ++k) {
            const int32_t v = it.srcs[k];
            auto f = pend_need.find(v);
            if (f == pend_need.end())
                pend_need.emplace(v, bit);
            else
                f->second |= bit;
            q->pending.push_back(v);
            if (q->sampled) q->mult[v] = it.mult[k];
        }
        q->outstanding = (int64_t)it.srcs.size();
        std::lock_guard<std::mutex> lk(mu);
        stats.admitted += 1;
        stats.active = nactive;
    }
    if (!deferred.empty()) {
        // back to the head of the queue, in their order (prepared again later)
        std::lock_guard<std::mutex> lk(mu);
        for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) queue.push_front(*it);
        defer_held = held_bytes;
    }
    return deferred.size() < prepq.size() || prepq.size() < batch.size();
}

// Runs one slice of tiles from the pending pool. Returns false when idle.
bool bc_server::run_slice_once() {
    if (nactive == 0) return false;
    const int S = 64 * bcd::tile_words_of(g);
    const int64_t cap = (int64_t)cfg.tiles_per_slice * S;
    std::vector<int32_t> take;
    std::vector<uint64_t> need;
    int idle_rounds = 0;
    while ((int64_t)take.size() < cap && idle_rounds < 64) {
        SQuery *q = slots[rr];
        rr = (rr + 1) & 63;
        if (!q || q->pending.empty()) {
            ++idle_rounds;
            continue;
        }
        idle_rounds = 0;
        // up to one tile's worth per query per round
        for (int k = 0; k < S && !q->pending.empty() && (int64_t)take.size() < cap; ++k) {
            const int32_t v = q->pending.front();
            q->pending.pop_front();
            auto f = pend_need.find(v);
            if (f == pend_need.end()) continue;  // already scheduled through another query
            take.push_back(v);
            need.push_back(f->second);
            pend_need.erase(f);
        }
    }
    if (take.empty()) {
        for (int s = 0; s < 64; ++s)
            if (slots[s] && slots[s]->outstanding <= 0) complete(slots[s], BC_OK);
        return false;
    }
    // tiles of sources at similar hop distance to the hub and of similar
    // two-hop reach (aligned levels)
    std::vector<size_t> order(take.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return bcd::source_order_key(g, take[a]) < bcd::source_order_key(g, take[b]);
    });
    const int64_t ntiles = ((int64_t)take.size() + S - 1) / S;
    std::vector<int32_t> srcs((size_t)ntiles * S, -1);
    std::vector<uint64_t> needs((size_t)ntiles * S, 0ull);
    uint64_t exact_q = 0, sampled_q = 0;
    for (int s = 0; s < 64; ++s)
        if (slots[s]) (slots[s]->sampled ? sampled_q : exact_q) |= 1ull << s;
    std::vector<uint32_t> mult;
    if (sampled_q) mult.assign((size_t)ntiles * S * 64, 0u);
    for (size_t i = 0; i < order.size(); ++i) {
        const size_t j = order[i];
        srcs[i] = take[j];
        needs[i] = need[j];
        uint64_t y = need[j] & sampled_q;
        while (y) {
            const int b = __builtin_ctzll(y);
            y &= y - 1;
            mult[i * 64 + b] = slots[b]->mult[take[j]];
        }
    }
    std::vector<double> partials;
    uint32_t qflags[64] = {0};
    unsigned long long edges = 0;
    const auto t0 = Clock::now();
    std::vector<int32_t> slot_roots(64, -1);
    for (int sl = 0; sl < 64; ++sl)
        if (slots[sl]) slot_roots[sl] = slots[sl]->q.r;
    bc_status st = bcd::run_slice(g, srcs, needs, mult, exact_q, slot_roots, partials, qflags, &edges);
    {
        std::lock_guard<std::mutex> lk(mu);
        stats.busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        stats.slices += 1;
        stats.sources_run += (int64_t)take.size();
        stats.edges_traversed += (int64_t)edges;
    }
    if (st != BC_OK) {
        fatal = st;
        fail_active(st);
        return true;
    }
    for (int s = 0; s < 64; ++s) {
        SQuery *q = slots[s];
        if (!q) continue;
        for (int64_t t = 0; t < ntiles; ++t) q->acc += partials[(size_t)t * 64 + s];
        if (qflags[s] & 1u) q->flags |= BC_FLAG_SIGMA_2_53;
    }
    for (size_t i = 0; i < take.size(); ++i) {
        uint64_t y = need[i];
        while (y) {
            const int b = __builtin_ctzll(y);
            y &= y - 1;
            if (slots[b]) slots[b]->outstanding -= 1;
        }
    }
    for (int s = 0; s < 64; ++s)
        if (slots[s] && slots[s]->outstanding <= 0) complete(slots[s], BC_OK);
    return true;
}

void bc_server::run() {
    cudaSetDevice(g->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            if (queue.empty() && nactive == 0) cv_work.wait_for(lk, std::chrono::milliseconds(20));
            if (stop) break;
        }
        bool did = admit();
        did = run_slice_once() || did;
        (void)did;
    }
    // fail whatever is left
    fail_active(BC_E_INTERNAL);
}

using namespace bcd;

extern "C" {

bc_status bc_server_create(bc_graph *g, const bc_server_config *cfg, bc_server **out) {
    if (!g || !out) return set_error(BC_E_INVALID_ARG, "bc_server_create: NULL argument");
    BCD_TRY(check_graph(g, "bc_server_create"));
    BCD_TRY(prepare_ordering(g));
    bc_server *s = new bc_server();
    s->g = g;
    s->cfg.max_active = 64;
    s->cfg.tiles_per_slice = 16;
    s->cfg.max_queue = 1 << 20;
    {
        // default budget: a quarter of the device memory free once the
        // graph's workspace exists
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = (size_t)1 << 30;
        }
        s->cfg.max_device_bytes = std::max<int64_t>((int64_t)(fr / 4), 1 << 20);
    }
    if (cfg) {
        if (cfg->max_active) s->cfg.max_active = cfg->max_active;
        if (cfg->tiles_per_slice) s->cfg.tiles_per_slice = cfg->tiles_per_slice;
        if (cfg->max_device_bytes) s->cfg.max_device_bytes = cfg->max_device_bytes;
        if (cfg->max_queue) s->cfg.max_queue = cfg->max_queue;
    }
    if (s->cfg.max_active < 1 || s->cfg.max_active > 64 || s->cfg.tiles_per_slice < 1 || s->cfg.max_queue < 1 ||
        s->cfg.max_device_bytes < 1) {
        delete s;
        return set_error(BC_E_INVALID_ARG, "bc_server_create: config out of range");
    }
    s->worker = std::thread([s]() { s->run(); });
    *out = s;
    return BC_OK;
}

bc_status bc_submit(bc_server *s, const bc_query *q, uint64_t *ticket) {
    if (!s || !q || !ticket) return set_error(BC_E_INVALID_ARG, "bc_submit: NULL argument");
    if (q->r < 0 || q->r >= s->g->n) return set_error(BC_E_INVALID_ARG, "bc_submit: query vertex out of range");
    SQuery *sq = new SQuery();
    sq->q = *q;
    if (q->kind == BC_QUERY_EXACT) {
    } else if (q->kind == BC_QUERY_APPROX) {
        if (!(q->eps > 0.0) || !(q->delta > 0.0 && q->delta < 1.0)) {
            delete sq;
            return set_error(BC_E_INVALID_ARG, "bc_submit: approx query needs eps > 0 and 0 < delta < 1");
        }
        const double T = samples_for(q->eps, q->delta);
        if (!(T >= 1.0) || T > 4.0e9) {
            delete sq;
            return set_error(BC_E_INVALID_ARG, "bc_submit: sample count out of range");
        }
        sq->T = (int64_t)T;
    } else if (q->kind == BC_QUERY_APPROX_T || q->kind == BC_QUERY_HYBRID) {
        if (q->T < 1 || q->T > 4000000000ll) {
            delete sq;
            return set_error(BC_E_INVALID_ARG, "bc_submit: T must be in [1, 4e9]");
        }
        sq->T = q->T;
    } else {
        delete sq;
        return set_error(BC_E_INVALID_ARG, "bc_submit: unknown query kind");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int64_t)s->queue.size() >= s->cfg.max_queue) {
        delete sq;
        return set_error(BC_E_BUSY, "bc_submit: queue full");
    }
    sq->ticket = s->next_ticket++;
    sq->t_submit = Clock::now();
    s->queue.push_back(sq);
    s->tickets[sq->ticket] = sq;
    s->stats.submitted += 1;
    *ticket = sq->ticket;
    s->cv_work.notify_one();
    return BC_OK;
}

bc_status bc_poll(bc_server *s, uint64_t ticket, bc_result *out, double *latency_ms, int64_t timeout_us) {
    if (!s || !out) return set_error(BC_E_INVALID_ARG, "bc_poll: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_error(BC_E_INVALID_ARG, "bc_poll: unknown ticket");
    SQuery *q = it->second;
    if (!q->done && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return q->done; });
    if (!q->done) return BC_E_PENDING;
    *out = q->res;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    s->tickets.erase(it);
    delete q;
    return BC_OK;
}

bc_status bc_server_stats_get(bc_server *s, bc_server_stats *st) {
    if (!s || !st) return set_error(BC_E_INVALID_ARG, "bc_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    st->queued = (int64_t)s->queue.size();
    return BC_OK;
}

void bc_server_destroy(bc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->tickets) delete kv.second;
    for (SQuery *q : s->queue)
        if (!s->tickets.count(q->ticket)) delete q;
    delete s;
}

}  // extern "C"
