// Weighted single-source work (Section 2 with positive integer weights, the
// SPD of each source) for a tile of S = 64 * nw sources (nw = 1, 2, 4, 8 or
// 16): exact distances in Dial's bucket order, sigma by a pull over tight
// in-arcs, and the dependencies of Eq. 4 by a pull over tight out-arcs.
//
// Distances are integers, so handling distance values in increasing order
// settles every (vertex, source) pair once, at its final distance: a
// relaxation that lowers dist_s(y) (atomicMin) queues the pair (y, s) in the
// ring slot of the new distance. The ring has R slots, R a power of two above
// the largest weight, so the distances in flight [d, d + R) never share a
// slot. Each slot is a circular buffer: entries between its consumed base and
// its count are pending. When slot d comes up, a pending pair whose distance
// still equals d is settled; a pair lowered since it was queued is stale and
// skipped. Every tight in-arc predecessor of a pair settled at d sits at a
// distance below d, so sigma_s(v) is complete when it is pulled.
//
// The unit of work is one (vertex, source) pair. Lanes take pairs, so a warp
// runs 32 independent chains of loads: a tile settles each vertex at as many
// distances as it has sources, and sources rarely share a distance. A pair
// whose vertex has more than 32 in- or out-arcs is cut into chunks of
// chunk_arcs arcs that warps take after a grid barrier (lanes over arcs);
// their sigma partial sums meet in fp64 atomic adds (integers: exact in any
// order below 2^53, and the running sum shows when 2^53 is passed).
//
// The backward pass walks the distance levels from the deepest, down to the
// shallowest level at which a query vertex sits for a source of the tile.
// Arc (v, y) is tight for s when dist_s(v) + w(v, y) = dist_s(y);
// c_s(y) = (1 + delta_s(y)) / sigma_s(y) replaces sigma in place. A short row
// is summed by one lane in CSR order, a long row per lane in a fixed arc
// order, then by a fixed butterfly per chunk, and the chunks are combined in
// chunk order by the last one to finish, so delta is run-to-run reproducible.
//
// Scan mode (every query of the launch at one vertex r) replaces the backward
// pass by one pass over the settled pairs: r lies on sigma_sr * sigma_rt of
// the sigma_st shortest s-t paths when d(s, r) + d(r, t) = d(s, t), so
// delta_s.(r) = sigma_sr * sum of sigma_rt / sigma_st over those t != s, r
// (the pair dependencies of Eq. 2), with d(r, t) and sigma_rt from an earlier
// scan-mode launch whose only source is r (kFlagRootOut).
#include "bcd_common.cuh"
#include "bcd_wcols.cuh"
#include "bcd_device.cuh"

namespace bcd {

namespace {

using namespace dev;

constexpr int kMaxWords = 16;  // largest tile: 1024 sources
constexpr double kTwo53 = 9007199254740992.0;

// Per-level counters of the weighted kernel: counter k of level l sits at
// lev_grab[k * (maxlev + 2) + l].
enum WLev : int {
    kGrabPairs = 0,    // forward: hand-out of 32-pair groups of the level's slot
    kChunksF = 1,      // forward: chunks of long rows emitted
    kGrabChunksF = 2,  // forward: hand-out of those chunks
    kGrabEntries = 3,  // backward: hand-out of 32-entry groups of the level
    kChunksB = 4,      // backward: chunks of long rows emitted
    kGrabChunksB = 5,  // backward: hand-out of those chunks
};

struct WStats {
    unsigned edges = 0, reached = 0, tight = 0, arcs = 0, vb = 0, eb = 0;
};

__device__ __forceinline__ void wflush(Counters *c, WStats &st, int lane) {
    unsigned long long v[6] = {st.edges, st.reached, st.tight, st.arcs, st.vb, st.eb};
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(kFull, v[i], o);
    if (lane == 0) {
        unsigned long long *dst[6] = {&c->edges, &c->reached, &c->tight, &c->arc_visits, &c->vb, &c->eb};
#pragma unroll
        for (int i = 0; i < 6; ++i)
            if (v[i]) atomicAdd(dst[i], v[i]);
    }
    st = WStats();
}

// Butterfly sum over the warp: every lane gets the same, order-fixed result.
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

struct Tile {
    int S;      // sources per tile
    int shift;  // log2(S)
};

// Queues the pair (y, s) at tentative distance nd (slot positions wrap
// around the slot's capacity; overflow is detected when the slot is read).
__device__ __forceinline__ void wenqueue(const TravParams &p, const Tile &t, int y, int s, unsigned long long nd) {
    const int slot = (int)(nd & (unsigned long long)(p.ring - 1));
    const unsigned long long pos = atomicAdd(&p.bcount[slot], 1ull);
    p.buckets[(size_t)slot * p.bcap + (size_t)(pos & (unsigned long long)(p.bcap - 1))] =
        ((uint32_t)y << t.shift) | (uint32_t)s;
}

// The graph arrays do not change during a launch, so their loads take the
// read-only path (cached in L1; a lane walking its own row reuses sectors).
// The per-arc loops handle arcs in groups of four whose loads are issued
// together; sums still run in arc order.
constexpr int kBatch = 4;

// Relaxes out-arcs a, a + step, ... < ae of a vertex settled at distance d for source s.
__device__ __forceinline__ void relax_row(const TravParams &p, const Tile &t, int s, unsigned long long d,
                                          long long a, long long ae, long long step) {
    for (; a < ae; a += kBatch * step) {
        int y[kBatch];
        unsigned long long nd[kBatch], cur[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const long long aj = a + j * step;
            y[j] = aj < ae ? __ldg(p.col + aj) : -1;
            nd[j] = aj < ae ? d + __ldg(p.wt + aj) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) cur[j] = y[j] >= 0 ? p.dist[((size_t)y[j] << t.shift) + s] : 0ull;
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            if (y[j] >= 0 && nd[j] < cur[j]) {
                unsigned long long *dp = reinterpret_cast<unsigned long long *>(p.dist + ((size_t)y[j] << t.shift) + s);
                const unsigned long long old = atomicMin(dp, nd[j]);
                if (nd[j] < old) wenqueue(p, t, y[j], s, nd[j]);
            }
        }
    }
}

// Sum of sigma_s(u) over the tight in-arcs among a, a + step, ... < ae of a
// vertex at distance d (u at distance d - w(u, v)).
__device__ __forceinline__ double pull_sigma(const TravParams &p, const Tile &t, int s, unsigned long long d,
                                             long long a, long long ae, long long step, unsigned &tight) {
    double acc = 0.0;
    for (; a < ae; a += kBatch * step) {
        size_t iu[kBatch];
        unsigned long long want[kBatch];
        bool ok[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const long long aj = a + j * step;
            const unsigned long long w = aj < ae ? __ldg(p.rwt + aj) : ~0ull;
            ok[j] = w <= d;
            iu[j] = ok[j] ? ((size_t)__ldg(p.rcol + aj) << t.shift) + s : 0;
            want[j] = d - w;
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) ok[j] = ok[j] && p.dist[iu[j]] == want[j];
        double v[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) v[j] = ok[j] ? p.sigma[iu[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < kBatch; ++j)
            if (ok[j]) {
                acc += v[j];
                tight += 1;
            }
    }
    return acc;
}

// Sum of c_s(y) over the tight out-arcs among a, a + step, ... < ae of a
// vertex at distance d.
__device__ __forceinline__ double pull_c(const TravParams &p, const Tile &t, int s, unsigned long long d, long long a,
                                         long long ae, long long step) {
    double acc = 0.0;
    for (; a < ae; a += kBatch * step) {
        size_t iy[kBatch];
        unsigned long long want[kBatch];
        bool ok[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const long long aj = a + j * step;
            ok[j] = aj < ae;
            iy[j] = ok[j] ? ((size_t)__ldg(p.col + aj) << t.shift) + s : 0;
            want[j] = ok[j] ? d + __ldg(p.wt + aj) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) ok[j] = ok[j] && p.dist[iy[j]] == want[j];
        double v[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) v[j] = ok[j] ? p.sigma[iy[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < kBatch; ++j)
            if (ok[j]) acc += v[j];
    }
    return acc;
}

// delta_s(v) from its sum of c over tight out-arcs; c_s(v) replaces sigma_s(v).
__device__ __forceinline__ void wfinalize(const TravParams &p, const Tile &t, const uint64_t *s_need, int v, int s,
                                          double acc) {
    double *sp = p.sigma + ((size_t)v << t.shift) + s;
    const double sv = *sp;
    const double dd = sv * acc;
    *sp = (1.0 + dd) / sv;
    const uint64_t qm = __ldg(p.qmask + v);
    if (qm) {
        uint64_t y = qm & s_need[s];
        while (y) {
            const int q = __ffsll((long long)y) - 1;
            y &= y - 1;
            p.dep[s * 64 + q] = dd;
        }
    }
}

__device__ __forceinline__ void flag_source(const TravParams &p, int s) {
    atomicOr(reinterpret_cast<unsigned long long *>(&p.srcflag[s >> 6]), 1ull << (s & 63));
}

// Writes the nch chunks of arcs [rb, re) (kind 0: out-arcs, 1: in-arcs) of
// history entry e; the source slot rides in the kind field.
__device__ __forceinline__ void emit_wchunks(const TravParams &p, long long c0, int v, int e, int s, int kind,
                                             long long rb, long long re, int nch) {
    const int CH = p.chunk_arcs;
    for (int k = 0; k < nch; ++k) {
        const long long a0 = rb + (long long)k * CH;
        store_chunk(&p.chunks[c0 + k], v, e, k, nch, a0, (int)(min(re, a0 + CH) - a0), kind | (s << 1));
    }
}

__global__ void __launch_bounds__(512, 2) wtrav_kernel(TravParams p) {
    const int lane = threadIdx.x & 31;
    const long long wpb = blockDim.x >> 5;
    const long long nwarps = (long long)gridDim.x * wpb;
    const long long gthr = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    __shared__ uint64_t s_need[64 * kMaxWords];
    __shared__ int32_t s_minql[64 * kMaxWords];
    __shared__ int32_t s_lstop;
    __shared__ int32_t s_k;
    Tile tl;
    tl.S = 64 * p.nw;
    tl.shift = 5 + __ffs(p.nw);
    const int S = tl.S;
    const int R = p.ring;
    const int CH = p.chunk_arcs;
    const long long LS = (long long)p.maxlev + 2;
    unsigned long long *wl = p.lev_grab;
    unsigned long long *bbase = p.bcount + R;  // consumed entries of each slot
    uint32_t gen = 0;
    WStats st;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_mark = timer ? global_ns() : 0ull;
    unsigned long long ns_fwd = 0, ns_bwd = 0, ns_other = 0;

    for (long long tile = 0; tile < p.ntiles; ++tile) {
        const int32_t *tsrc = p.srcs + tile * S;
        check_cancel(p);
        if (blockIdx.x == 0) {
            for (int t = threadIdx.x; t < S; t += blockDim.x) {
                const int v = tsrc[t];
                if (v >= 0) {
                    p.dist[((size_t)v << tl.shift) + t] = 0ull;
                    wenqueue(p, tl, v, t, 0ull);
                }
            }
            for (int i = threadIdx.x; i < S * 64; i += blockDim.x) p.qlevel[i] = -1;
            for (int i = threadIdx.x; i < p.nw; i += blockDim.x) p.srcflag[i] = 0ull;
            if (p.mode == kModeScan)
                for (int i = threadIdx.x; i < 2 * S; i += blockDim.x) p.vsum[i] = 0.0;
            if (p.mode == kModeScan && p.ncols >= 2)
                for (int i = threadIdx.x; i < S * 64; i += blockDim.x) p.msum[i] = 0.0;
        }
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const int32_t v = tsrc[s];
            s_need[s] = v >= 0 ? p.need[v] : 0ull;
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
        }

        // ---------------- forward: settle distance values in order ----------------
        long long d = 0, es = 0;
        int seg = 0;
        bool first = true;
        for (;;) {
            // next slot with pending entries (every block finds the same one)
            if (threadIdx.x == 0) s_k = R;
            __syncthreads();
            for (int k = threadIdx.x + (first ? 0 : 1); k < R; k += blockDim.x) {
                const int sl = (int)((d + k) & (R - 1));
                if (ld_vol(&p.bcount[sl]) > ld_vol(&bbase[sl])) {
                    atomicMin(&s_k, k);
                    break;
                }
            }
            __syncthreads();
            const int kmin = s_k;
            __syncthreads();
            if (kmin >= R) break;
            first = false;
            if (seg + 2 > p.maxlev) {
                if (threadIdx.x == 0) set_err(p.ctr, kDevLevelOverflow);
                return;
            }
            d += kmin;
            const unsigned long long du = (unsigned long long)d;
            const int slot = (int)(d & (R - 1));
            const unsigned long long b0 = ld_vol(&bbase[slot]);
            long long cnt = (long long)(ld_vol(&p.bcount[slot]) - b0);
            if (cnt > p.bcap) {
                if (threadIdx.x == 0) set_err(p.ctr, kDevBucketOverflow);
                cnt = 0;
            }
            const uint32_t *bk = p.buckets + (size_t)slot * p.bcap;
            // the level's start and distance are recorded before the barrier
            // that ends step 1: the backward pass may follow the last level
            // with no other barrier in between
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                p.lev_start[seg] = es;
                p.lev_dist[seg] = d;
            }
            // step 1: the slot's pairs; short rows finish here. A pair gets
            // LPP lanes (1, 2, 4 or 8: the most with which the level's pairs
            // still fit the grid's lanes once), each walking every LPP-th arc
            // of its rows, so a level with few pairs does not wait on one lane
            // walking a whole row; the subgroup's sigma parts meet in a fixed
            // shuffle tree (integers: exact).
            {
                int LPP = 1;
                while (LPP < 8 && cnt * (long long)(2 * LPP) <= 32 * nwarps) LPP <<= 1;
                const int per = 32 / LPP;  // pairs per warp step
                const int sub = lane / LPP, rl = lane % LPP;
                const bool lead = rl == 0;
                ChunkGrabber grab(&wl[kGrabPairs * LS + seg], (cnt + per - 1) / per, nwarps);
                long long gi;
                while (grab.next(gi, lane)) {
                    const long long i = gi * per + sub;
                    int x = 0, s = 0;
                    bool ok = false;
                    if (i < cnt) {
                        const uint32_t pk = bk[(b0 + (unsigned long long)i) & (unsigned long long)(p.bcap - 1)];
                        x = (int)(pk >> tl.shift);
                        s = (int)(pk & (uint32_t)(S - 1));
                        ok = p.dist[((size_t)x << tl.shift) + s] == du;
                    }
                    const unsigned am = __ballot_sync(kFull, ok && lead);
                    if (am == 0u) continue;
                    unsigned long long eb = 0;
                    if (lane == 0) eb = atomicAdd(&p.lev_cnt[seg], (unsigned long long)__popc(am));
                    eb = __shfl_sync(kFull, eb, 0);
                    const long long e = es + (long long)eb + __popc(am & ((1u << (sub * LPP)) - 1u));
                    bool go = ok;
                    if (go && e >= p.hcap) {
                        if (lead) set_err(p.ctr, kDevHistOverflow);
                        go = false;
                    }
                    long long rb = 0, re = 0, irb = 0, ire = 0;
                    if (go) {
                        rb = __ldg(p.off + x);
                        re = __ldg(p.off + x + 1);
                        irb = __ldg(p.roff + x);
                        ire = d > 0 ? __ldg(p.roff + x + 1) : irb;
                    }
                    if (go && lead) {
                        p.hv[e] = x;
                        p.hs[e] = (uint16_t)s;
                        st.reached += 1;
                        st.edges += (unsigned)(re - rb);
                        if (atomicCAS(&p.tag[x], -1, 0) == -1) {
                            st.vb += 1;
                            st.eb += (unsigned)(re - rb);
                        }
                        const uint64_t qm = __ldg(p.qmask + x);
                        if (qm) {
                            uint64_t y = qm & s_need[s];
                            while (y) {
                                const int q = __ffsll((long long)y) - 1;
                                y &= y - 1;
                                p.qlevel[s * 64 + q] = seg;
                            }
                        }
                    }
                    const bool shortrow = go && re - rb <= p.wshort && ire - irb <= p.wshort;
                    double part = 0.0;
                    if (shortrow && d > 0) part = pull_sigma(p, tl, s, du, irb + rl, ire, LPP, st.tight);
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1)
                        if (o < LPP) part += __shfl_xor_sync(kFull, part, o);
                    double *sp = p.sigma + ((size_t)x << tl.shift) + s;
                    if (shortrow) {
                        if (lead) {
                            const double sg = d > 0 ? part : 1.0;
                            *sp = sg;
                            if (sg >= kTwo53) flag_source(p, s);
                            st.arcs += (unsigned)((re - rb) + (ire - irb));
                        }
                        relax_row(p, tl, s, du, rb + rl, re, LPP);
                    } else if (go && lead) {
                        if (d == 0) *sp = 1.0;
                        const int nin = (int)((ire - irb + CH - 1) / CH);
                        const int nout = (int)((re - rb + CH - 1) / CH);
                        const long long c0 =
                            (long long)atomicAdd(&wl[kChunksF * LS + seg], (unsigned long long)(nin + nout));
                        if (c0 + nin + nout > p.ccap) {
                            set_err(p.ctr, kDevChunkOverflow);
                        } else {
                            emit_wchunks(p, c0, x, (int)e, s, 1, irb, ire, nin);
                            emit_wchunks(p, c0 + nin, x, (int)e, s, 0, rb, re, nout);
                        }
                    }
                }
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            const long long ecnt = (long long)ld_vol(&p.lev_cnt[seg]);
            const long long ccnt = (long long)ld_vol(&wl[kChunksF * LS + seg]);
            // every block has read the slot's base by now; the new base is
            // next read R distances later, many barriers on
            if (blockIdx.x == 0 && threadIdx.x == 0) bbase[slot] = b0 + (unsigned long long)cnt;
            // step 2: chunks of long rows (lanes over arcs)
            if (ccnt > 0) {
                ChunkGrabber grab(&wl[kGrabChunksF * LS + seg], ccnt, nwarps);
                long long c;
                while (grab.next(c, lane)) {
                    const Chunk ch = load_chunk(&p.chunks[c]);
                    const int s = ch.pad >> 1;
                    if (ch.pad & 1) {
                        const double part = pull_sigma(p, tl, s, du, ch.a0 + lane, ch.a0 + ch.na, 32, st.tight);
                        const double sum = warp_sum(part);
                        if (lane == 0) {
                            const double old = atomicAdd(p.sigma + ((size_t)ch.v << tl.shift) + s, sum);
                            if (old + sum >= kTwo53) flag_source(p, s);
                        }
                    } else {
                        relax_row(p, tl, s, du, ch.a0 + lane, ch.a0 + ch.na, 32);
                    }
                    if (lane < ch.na) st.arcs += (unsigned)((ch.na - lane + 31) / 32);
                }
                if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            }
            es += ecnt;
            ++seg;
        }
        const int nseg = seg;
        const long long total = es;
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicMax(&p.ctr->levels_max, (unsigned long long)(nseg > 0 ? nseg - 1 : 0));
        if (timer) {
            const unsigned long long t = global_ns();
            ns_fwd += t - t_mark;
            t_mark = t;
        }

        // ---------------- the query vertex's own traversal ----------------
        if (p.mode == kModeScan && (p.flags & kFlagRootOut)) {
            // source slot 0 is r: keep d(r, t) and sigma_rt; with several query
            // vertices, slot c is column c
            for (long long e = gthr; e < total; e += nthr) {
                const int v = p.hv[e];
                const int c = p.hs[e];
                const size_t iv = ((size_t)v << tl.shift) + c;
                if (p.ncols >= 2) {
                    p.rdistq[(size_t)v * wcols_stride(p.ncols) + c] = p.dist[iv];
                    p.rsigq[(size_t)v * wcols_stride(p.ncols) + c] = p.sigma[iv];
                } else {
                    p.rdist[v] = p.dist[iv];
                    p.rsig[v] = p.sigma[iv];
                }
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        }
        // ---------------- vertex scan, several query vertices ----------------
        // Column c (query vertex r_c) of a settled pair (t, s) of distance D
        // takes sigma_{r_c t} / sigma_st when d(s, r_c) + d(r_c, t) = D with
        // d(r_c, t) >= 1, for the columns of the queries that need s; the terms
        // meet in msum[s * 64 + c] by fp64 atomic adds. Block 0 keeps
        // sigma_s(r_c) in msum[S * 64 + s * 64 + c] before the closing barrier
        // (the tile-end reset clears sigma).
        if (p.mode == kModeScan && p.ncols >= 2 && !(p.flags & (kFlagRootOut | kFlagNoBackward))) {
            unsigned pairs = 0;
            for (int sg = 1; sg < nseg; ++sg) {
                const long long e0 = p.lev_start[sg];
                const long long ne = (long long)p.lev_cnt[sg];
                const unsigned long long dk = (unsigned long long)p.lev_dist[sg];
                for (long long i = gthr; i < ne; i += nthr) {
                    const long long e = e0 + i;
                    const int t = p.hv[e];
                    const int s = p.hs[e];
                    uint64_t x = s_need[s];
                    uint64_t done = 0ull;
                    double sst = 0.0;
                    while (x) {
                        const int q = __ffsll((long long)x) - 1;
                        x &= x - 1;
                        const int c = p.qcol[q];
                        if ((done >> c) & 1ull) continue;
                        done |= 1ull << c;
                        const int ql = p.qlevel[s * 64 + q];
                        if (ql < 0) continue;
                        const unsigned long long rd = p.rdistq[(size_t)t * wcols_stride(p.ncols) + c];
                        if (rd == 0ull || rd >= dk) continue;  // t = r_c, unreached from r_c, or too far
                        if ((unsigned long long)p.lev_dist[ql] + rd != dk) continue;
                        if (sst == 0.0) sst = p.sigma[((size_t)t << tl.shift) + s];
                        atomicAdd(&p.msum[s * 64 + c], p.rsigq[(size_t)t * wcols_stride(p.ncols) + c] / sst);
                        ++pairs;
                    }
                }
            }
            if (blockIdx.x == 0) {
                for (int i = threadIdx.x; i < S * 64; i += blockDim.x) {
                    const int s = i >> 6, q = i & 63;
                    if (!((s_need[s] >> q) & 1ull)) continue;
                    const int c = p.qcol[q];
                    p.msum[(size_t)S * 64 + s * 64 + c] = p.sigma[((size_t)p.croot[c] << tl.shift) + s];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
            if (lane == 0 && pairs) atomicAdd(&p.ctr->vpairs, (unsigned long long)pairs);
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        }
        // ---------------- vertex scan over the settled pairs ----------------
        // A settled pair (t, s) of level sg (distance D) takes the term
        // sigma_rt / sigma_st when d(s, r) + d(r, t) = D, with d(r, t) >= 1
        // (t != r). d(s, r) is the distance of the level at which r settled
        // for s (its query level). Terms meet in vsum[s] by fp64 atomic adds;
        // block 0 keeps sigma_sr in vsum[S + s] before the closing barrier.
        if (p.mode == kModeScan && p.ncols < 2 && !(p.flags & (kFlagRootOut | kFlagNoBackward))) {
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                const uint64_t x = s_need[s];
                const int qs = x ? p.qlevel[s * 64 + __ffsll((long long)x) - 1] : -1;
                s_minql[s] = qs;
                if (blockIdx.x == 0) p.vsum[S + s] = qs >= 0 ? p.sigma[((size_t)p.vroot << tl.shift) + s] : 0.0;
            }
            __syncthreads();
            unsigned pairs = 0;
            for (int sg = 1; sg < nseg; ++sg) {
                const long long e0 = p.lev_start[sg];
                const long long ne = (long long)p.lev_cnt[sg];
                const unsigned long long dk = (unsigned long long)p.lev_dist[sg];
                for (long long i = gthr; i < ne; i += nthr) {
                    const long long e = e0 + i;
                    const int v = p.hv[e];
                    const unsigned long long rd = p.rdist[v];
                    if (rd == 0ull || rd >= dk) continue;  // t = r, t unreached from r, or d(s, r) < 1
                    const int s = p.hs[e];
                    const int qs = s_minql[s];
                    if (qs < 0 || (unsigned long long)p.lev_dist[qs] + rd != dk) continue;
                    atomicAdd(&p.vsum[s], p.rsig[v] / p.sigma[((size_t)v << tl.shift) + s]);
                    ++pairs;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
            if (lane == 0 && pairs) atomicAdd(&p.ctr->vpairs, (unsigned long long)pairs);
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        }

        // ---------------- backward (Eq. 4) over the levels ----------------
        if (p.mode == kModeSpd && !(p.flags & kFlagNoBackward)) {
            if (threadIdx.x == 0) s_lstop = 0x7fffffff;
            __syncthreads();
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                int mq = 0x7fffffff;
                if (tsrc[s] >= 0) {
                    if (p.flags & kFlagFullBackward) {
                        mq = 0;
                    } else {
                        uint64_t y = s_need[s];
                        while (y) {
                            const int q = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            const int lv = p.qlevel[s * 64 + q];
                            if (lv >= 0 && lv < mq) mq = lv;
                        }
                    }
                }
                s_minql[s] = mq;
                atomicMin(&s_lstop, mq);
            }
            __syncthreads();
            const int lstop = s_lstop;
            for (int sg = nseg - 1; sg >= lstop && lstop < nseg; --sg) {
                const long long e0 = p.lev_start[sg];
                const long long ne = (long long)p.lev_cnt[sg];
                const unsigned long long dk = (unsigned long long)p.lev_dist[sg];
                // step 1: the level's entries, one per lane; short rows finish here
                {
                    ChunkGrabber grab(&wl[kGrabEntries * LS + sg], (ne + 31) / 32, nwarps);
                    long long gi;
                    while (grab.next(gi, lane)) {
                        const long long i = gi * 32 + lane;
                        if (i >= ne) continue;
                        const long long e = e0 + i;
                        const int s = p.hs[e];
                        if (s_minql[s] > sg) continue;
                        const int v = p.hv[e];
                        const long long rb = __ldg(p.off + v), re = __ldg(p.off + v + 1);
                        if (re - rb <= p.wshort) {
                            const double acc = pull_c(p, tl, s, dk, rb, re, 1);
                            wfinalize(p, tl, s_need, v, s, acc);
                            st.arcs += (unsigned)(re - rb);
                        } else {
                            const int nch = (int)((re - rb + CH - 1) / CH);
                            const long long c0 =
                                (long long)atomicAdd(&wl[kChunksB * LS + sg], (unsigned long long)nch);
                            if (c0 + nch > p.ccap || c0 + nch > p.pcap)
                                set_err(p.ctr, kDevChunkOverflow);
                            else
                                emit_wchunks(p, c0, v, (int)e, s, 0, rb, re, nch);
                        }
                    }
                }
                if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
                const long long ccnt = (long long)ld_vol(&wl[kChunksB * LS + sg]);
                // step 2: chunks of long rows (partial sums indexed by chunk;
                // an entry's chunks are consecutive); the last chunk of an
                // entry to finish combines them in chunk order
                if (ccnt > 0) {
                    ChunkGrabber grab(&wl[kGrabChunksB * LS + sg], ccnt, nwarps);
                    long long c;
                    while (grab.next(c, lane)) {
                        const Chunk ch = load_chunk(&p.chunks[c]);
                        const int s = ch.pad >> 1;
                        const double part = pull_c(p, tl, s, dk, ch.a0 + lane, ch.a0 + ch.na, 32);
                        const double sum = warp_sum(part);
                        if (lane < ch.na) st.arcs += (unsigned)((ch.na - lane + 31) / 32);
                        if (lane == 0) {
                            const long long base = c - ch.k;
                            __stcg(&p.partial[c], sum);
                            __threadfence();
                            const int prev = atomicAdd(&p.pdone[base], 1);
                            if (prev == ch.nch - 1) {
                                __threadfence();
                                double acc = 0.0;
                                for (int k = 0; k < ch.nch; ++k) acc += __ldcg(&p.partial[base + k]);
                                p.pdone[base] = 0;
                                wfinalize(p, tl, s_need, ch.v, s, acc);
                            }
                        }
                    }
                    if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
                }
            }
        }
        if (timer) {
            const unsigned long long t = global_ns();
            ns_bwd += t - t_mark;
            t_mark = t;
        }
        wflush(p.ctr, st, lane);

        // ---------------- tile end ----------------
        if (p.mode == kModeScan && blockIdx.x == 0) {
            // one value per source (one query vertex) or per (source, column)
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                uint64_t x = s_need[s];
                const double dv = p.vsum[S + s] * p.vsum[s];
                while (x) {
                    const int q = __ffsll((long long)x) - 1;
                    x &= x - 1;
                    if (p.ncols >= 2) {
                        const int c = p.qcol[q];
                        p.dep[s * 64 + q] = p.msum[(size_t)S * 64 + s * 64 + c] * p.msum[s * 64 + c];
                    } else {
                        p.dep[s * 64 + q] = dv;
                    }
                }
            }
            __syncthreads();
        }
        if (blockIdx.x == 0) tile_query_sums(p, tile, S, tsrc, s_need);
        if (!(p.flags & kFlagNoReset)) {
            for (long long e = gthr; e < total; e += nthr) {
                const int v = p.hv[e];
                const size_t iv = ((size_t)v << tl.shift) + p.hs[e];
                p.sigma[iv] = 0.0;
                p.dist[iv] = ~0ull;
                p.tag[v] = -1;
            }
            if (blockIdx.x == 0) {
                for (int l = threadIdx.x; l <= nseg + 1; l += blockDim.x) {
                    p.lev_cnt[l] = 0ull;
#pragma unroll
                    for (int k = 0; k < 6; ++k) wl[k * LS + l] = 0ull;
                }
                for (int i = threadIdx.x; i < 2 * R; i += blockDim.x) p.bcount[i] = 0ull;
            }
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
        }
    }
    if (timer) {
        p.ctr->ns_fwd += ns_fwd;
        p.ctr->ns_bwd += ns_bwd;
        p.ctr->ns_other += ns_other;
    }
}

}  // namespace

bc_status launch_weighted(bc_graph *g, TravParams &p) {
    const int threads = g->block_threads;
    int per_sm = 0;
    BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wtrav_kernel, threads, 0));
    if (per_sm < 1) return set_error(BC_E_INTERNAL, "weighted traversal kernel cannot be resident");
    dim3 grid((unsigned)(g->num_sms * per_sm)), block((unsigned)threads);
    void *args[] = {(void *)&p};
    BCD_CUDA(cudaLaunchCooperativeKernel((const void *)wtrav_kernel, grid, block, args, 0, g->stream));
    g->launches += 1;
    g->last_grid = (int)grid.x;
    return BC_OK;
}

}  // namespace bcd
