// Weighted single-source work (Section 2 with positive integer weights) with
// one source per block: each block takes the next source of the launch's
// union, runs its SPD in Dial's bucket order with block-wide barriers only,
// accumulates its dependencies (Eq. 4, or the vertex scan), writes them and
// takes the next source. Blocks never wait on one another, so a block whose
// source is cheap moves on while another is still deep in its distances:
// the grid-wide barrier per distance value of the tile kernel (hundreds of
// them per tile with weights up to 255) is gone, and so is the idle time of
// every lane waiting there for the slowest chain of the level.
//
// State of a block, for its current source s: one (dist(v), sigma(v)) pair
// per vertex v, 16 bytes (distance all ones when unreached; during the Eq. 4
// pass c(v) = (1 + delta(v)) / sigma(v) replaces sigma in place) or, in
// vertex-scan launches, one 8-byte word (24-bit distance, 40-bit count: half
// the footprint, so more of it stays in L2; a launch that overflows them
// reruns on 16-byte pairs); the settled vertices in settling order (history)
// with the start and distance of each distance level; and the bucket ring: R
// slots (R a power of two above the largest weight) of bcap queued vertices
// each, with their queued / consumed counters in shared memory. Eq. 4
// launches also keep one bit per arc (see src_relax).
//
// Sigma rides along the relaxations. Settling u at distance d (its sigma is
// final: every predecessor on a shortest path sits at a smaller distance and
// relaxed its arcs in an earlier level), each out-arc (u, v, w) offers the
// candidate nd = d + w: if nd is below dist(v) the pair becomes (nd,
// sigma(u)) and v is queued in the slot of nd; if nd equals dist(v),
// sigma(u) is added. The pair changes by one compare-and-swap (128 or 64
// bits), so a distance and its path count always move together, and when v settles its
// pair holds its distance with the sum over exactly its tight in-arcs (sigma
// values are integers: exact in any order below 2^53). Every arc is read
// once in the forward pass, along its tail's out-row; no in-arc pass.
// A vertex queued in the slot of d whose distance has since dropped is stale
// and skipped; a vertex is queued only when its distance strictly drops, so
// it settles once.
//
// A level's queued vertices are spread over the block's lanes, 1 to 32 lanes
// per vertex (as many as the level's size leaves room for); each lane walks
// every LPP-th arc. Vertices with more than weighted_short_row out-arcs are
// cut into chunk_arcs chunks that warps take after a block barrier (lanes
// over arcs). The source is flagged when a sigma reaches 2^53. The Eq. 4
// pass walks the levels from the deepest to the shallowest level holding a
// query vertex the source serves, summing c over tight out-arcs (short rows
// by LPP lanes and a fixed shuffle tree, long rows by chunks added in chunk
// order), so delta is the same from run to run.
//
// Each source's dependencies delta_s.(r_q) go to sdep[i * 64 + q] (i its
// position in the launch's source list, q the queries that need it); a
// second kernel forms the per-tile, per-query sums in the fixed order the
// tile kernel uses.
//
// Bounded work: no block ever waits on another. A source that runs longer
// than timeout_ns, a full bucket slot, level array or chunk list, or a cancel
// request sets the launch's error word; the block leaves, the others stop at
// their next source, and the host resets the state (and grows what was full).
#include "bcd_common.cuh"
#include "bcd_wcols.cuh"
#include "bcd_device.cuh"

namespace bcd {

namespace {

using namespace dev;

constexpr int kLanesBatch = 4;  // arcs a lane loads together
// One block of 1024 threads per SM: fewer sources in flight, each with more
// lanes, measured faster than two blocks of 512 or four of 256 (a smaller
// footprint of per-source state, and shorter per-level chains)
constexpr int kSrcThreads = 1024;
constexpr double kSrcTwo53 = 9007199254740992.0;

// (distance, sigma) of one vertex for the block's current source
struct __align__(16) DistSig {
    unsigned long long d;
    double s;
};

struct SrcParams {
    DistSig *ds;                // [blocks * n]
    int32_t *hv;                // [blocks * n] settled vertices of the current source
    int32_t *lstart;            // [blocks * maxlev] first history entry of each level
    unsigned long long *ldist;  // [blocks * maxlev] distance of each level
    uint32_t *bk;               // [blocks * ring * bcap] queued vertices, circular per slot
    Chunk *ch;                  // [blocks * chcap] long-row chunks of one level
    double *part;               // [blocks * chcap] backward chunk sums
    uint32_t *tb;               // [blocks * tbw] one bit per arc: its offer took effect (Eq. 4 launches)
    int64_t tbw;                // words per block: (m + 31) / 32
    double *sdep;               // [nsrc * 64]
    uint32_t *sflag;            // [nsrc] sigma >= 2^53 seen
    unsigned long long *next;   // source hand-out
    int64_t n;
    int64_t bcap;               // power of two
    int64_t chcap;
    int64_t nsrc;               // ntiles * S (padding entries are -1)
    int32_t ring;
    int32_t maxlev;
};

struct SrcStats {
    unsigned long long edges = 0, reached = 0, tight = 0, arcs = 0, vb = 0, eb = 0, pairs = 0;
};

__device__ __forceinline__ double sum_warp(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// 16-byte compare-and-swap of a (distance, sigma) pair: true when *p held
// `expect` and now holds `nw`; otherwise `expect` receives what *p held.
__device__ __forceinline__ bool cas_pair(DistSig *p, DistSig &expect, const DistSig &nw) {
    const unsigned long long e0 = expect.d, e1 = (unsigned long long)__double_as_longlong(expect.s);
    const unsigned long long n0 = nw.d, n1 = (unsigned long long)__double_as_longlong(nw.s);
    unsigned long long o0, o1;
    asm volatile(
        "{\n\t.reg .b128 e, n, o;\n\t"
        "mov.b128 e, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], e, n;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(o0), "=l"(o1)
        : "l"(e0), "l"(e1), "l"(n0), "l"(n1), "l"(p)
        : "memory");
    const bool ok = o0 == e0 && o1 == e1;
    expect.d = o0;
    expect.s = __longlong_as_double((long long)o1);
    return ok;
}

constexpr int kCasTries = 1 << 16;  // a pair changed under us this often: give up (never seen)

// Outcome of one offer to a head's pair.
enum Offer : int { kOfferNone = 0, kOfferTie = 1, kOfferLower = 2, kOfferStuck = -1, kOfferWide = -2 };

// Wide layout: 16-byte (distance, sigma) pairs, sigma in fp64 (the Eq. 4
// pass stores c there). Needed for Eq. 4 launches and for counts of 2^40 and
// more.
struct WidePairs {
    static constexpr bool kWide = true;
    static constexpr unsigned long long kUnreached = ~0ull;
    DistSig *ds;
    __device__ __forceinline__ unsigned long long dist(int v) const { return ds[v].d; }
    __device__ __forceinline__ void get(int v, unsigned long long &d, double &sg) const {
        const DistSig x = ds[v];
        d = x.d;
        sg = x.s;
    }
    __device__ __forceinline__ void seed(int v) const {
        DistSig x;
        x.d = 0ull;
        x.s = 1.0;
        ds[v] = x;
    }
    __device__ __forceinline__ void clear(int v) const {
        DistSig x;
        x.d = ~0ull;
        x.s = 0.0;
        ds[v] = x;
    }
    __device__ __forceinline__ int offer(int v, unsigned long long nd, double sg) const {
        DistSig *q = ds + v;
        DistSig cur = *q;
        for (int it = 0; it < kCasTries; ++it) {
            if (nd > cur.d) return kOfferNone;
            const bool lower = nd < cur.d;
            DistSig nw;
            nw.d = nd;
            nw.s = lower ? sg : cur.s + sg;
            if (cas_pair(q, cur, nw)) return lower ? kOfferLower : kOfferTie;
        }
        return kOfferStuck;
    }
};

// Narrow layout: one 8-byte word per vertex, the distance in bits 0-23
// (2^24 - 1: unreached) and sigma as an integer in bits 24-63, changed by a
// 64-bit compare-and-swap. Half the footprint of the wide pairs, so more of
// the block's state stays in L2. A distance of 2^24 - 1 or more, or a count
// of 2^40 or more, asks for the wide layout (the launch reruns with it).
struct NarrowPairs {
    static constexpr bool kWide = false;
    static constexpr unsigned long long kDistMask = (1ull << 24) - 1;
    static constexpr unsigned long long kUnreached = kDistMask;
    static constexpr unsigned long long kSigLimit = 1ull << 40;
    unsigned long long *w;
    __device__ __forceinline__ unsigned long long dist(int v) const { return w[v] & kDistMask; }
    __device__ __forceinline__ void get(int v, unsigned long long &d, double &sg) const {
        const unsigned long long x = w[v];
        d = x & kDistMask;
        sg = (double)(x >> 24);
    }
    __device__ __forceinline__ void seed(int v) const { w[v] = 1ull << 24; }
    __device__ __forceinline__ void clear(int v) const { w[v] = kDistMask; }
    __device__ __forceinline__ int offer(int v, unsigned long long nd, double sg) const {
        if (nd >= kDistMask) return kOfferWide;
        const unsigned long long si = (unsigned long long)sg;  // an integer below 2^40
        unsigned long long cur = w[v];
        for (int it = 0; it < kCasTries; ++it) {
            const unsigned long long cd = cur & kDistMask;
            if (nd > cd) return kOfferNone;
            const bool lower = nd < cd;
            const unsigned long long ns = lower ? si : (cur >> 24) + si;
            if (ns >= kSigLimit) return kOfferWide;
            const unsigned long long nw = nd | (ns << 24);
            const unsigned long long old = atomicCAS(w + v, cur, nw);
            if (old == cur) return lower ? kOfferLower : kOfferTie;
            cur = old;
        }
        return kOfferStuck;
    }
};

// Offers out-arcs a, a + step, ... < ae of a vertex settled at distance d
// with path count sg: lowers a head's distance (and queues it) or adds sg to
// its count when the candidate ties. With tb (Eq. 4 launches), an offer that
// took effect also sets its arc's bit: every tight arc gets one (its offer
// of the final distance always takes effect), and arcs whose offer a shorter
// path replaced keep a stale bit that the backward's check drops. Returns 0,
// or the device error to raise (a pair that kept changing, a count or
// distance the narrow layout cannot hold).
template <class PairT>
__device__ __forceinline__ int src_relax(const TravParams &p, const PairT &P, uint32_t *bk, uint32_t *s_cnt,
                                         uint32_t *tb, int64_t bcap, int R, unsigned long long d, double sg,
                                         long long a, long long ae, int step, unsigned long long &adds) {
    int err = 0;
    for (; a < ae; a += kLanesBatch * step) {
        int y[kLanesBatch];
        unsigned long long nd[kLanesBatch], cd[kLanesBatch];
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j) {
            const long long aj = a + (long long)j * step;
            y[j] = aj < ae ? __ldg(p.col + aj) : -1;
            nd[j] = aj < ae ? d + __ldg(p.wt + aj) : 0ull;
        }
        // the heads' distances first; the compare-and-swap only for the few
        // candidates that lower or tie
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j) cd[j] = y[j] >= 0 ? P.dist(y[j]) : 0ull;
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j) {
            if (y[j] < 0 || nd[j] > cd[j]) continue;
            const int r = P.offer(y[j], nd[j], sg);
            if (r > 0) {
                adds += 1;
                if (tb) {
                    const long long aj = a + (long long)j * step;
                    atomicOr(tb + (aj >> 5), 1u << (aj & 31));
                }
                if (r == kOfferLower) {
                    const int slot = (int)(nd[j] & (unsigned long long)(R - 1));
                    const uint32_t pos = atomicAdd(&s_cnt[slot], 1u);
                    bk[(size_t)slot * (size_t)bcap + (pos & (uint32_t)(bcap - 1))] = (uint32_t)y[j];
                }
            } else if (r == kOfferStuck) {
                err = kDevTimeout;
            } else if (r == kOfferWide) {
                err = kDevWide;
            }
        }
    }
    return err;
}

// Sum of c(y) over the tight out-arcs (y at distance d + w(v, y)) among a,
// a + step, ... < ae of a vertex at distance d. Only arcs whose bit the
// forward set can be tight; the others are skipped without reading their
// head.
__device__ __forceinline__ double src_pull_c(const TravParams &p, const DistSig *ds, const uint32_t *tb,
                                             unsigned long long d, long long a, long long ae, int step) {
    double acc = 0.0;
    for (; a < ae; a += kLanesBatch * step) {
        int y[kLanesBatch];
        unsigned long long want[kLanesBatch];
        bool ok[kLanesBatch];
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j) {
            const long long aj = a + (long long)j * step;
            ok[j] = aj < ae && ((tb[aj >> 5] >> (aj & 31)) & 1u);
            y[j] = ok[j] ? __ldg(p.col + aj) : 0;
            want[j] = ok[j] ? d + __ldg(p.wt + aj) : 0ull;
        }
        DistSig v[kLanesBatch];
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j) {
            if (ok[j]) {
                v[j] = ds[y[j]];
            } else {
                v[j].d = ~0ull;
                v[j].s = 0.0;
            }
        }
#pragma unroll
        for (int j = 0; j < kLanesBatch; ++j)
            if (ok[j] && v[j].d == want[j]) acc += v[j].s;
    }
    return acc;
}

// Lanes per vertex for a level of cnt vertices on a block of bd threads: the
// most (up to a warp) with which every vertex still gets its lanes at once.
__device__ __forceinline__ int lanes_per_vertex(long long cnt, int bd) {
    int lpp = 1;
    while (lpp < 32 && cnt * (long long)(2 * lpp) <= (long long)bd) lpp <<= 1;
    return lpp;
}

// Sum of the lane parts of one vertex's LPP lanes (a fixed butterfly).
__device__ __forceinline__ double sum_lanes(double x, int lpp) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1)
        if (o < lpp) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ void src_store_chunks(Chunk *chs, long long c0, int v, int e, int kind, long long rb,
                                                 long long re, int nch, int CH) {
    for (int k = 0; k < nch; ++k) {
        const long long a0 = rb + (long long)k * CH;
        store_chunk(&chs[c0 + k], v, e, k, nch, a0, (int)(min(re, a0 + CH) - a0), kind);
    }
}

// delta(v) = sigma(v) * acc; c(v) = (1 + delta(v)) / sigma(v) replaces sigma(v).
__device__ __forceinline__ void src_finalize(const TravParams &p, DistSig *ds, uint64_t need, double *s_dep, int v,
                                             double acc) {
    const double sv = ds[v].s;
    const double dd = sv * acc;
    ds[v].s = (1.0 + dd) / sv;
    uint64_t y = __ldg(p.qmask + v) & need;
    while (y) {
        const int q = __ffsll((long long)y) - 1;
        y &= y - 1;
        s_dep[q] = dd;
    }
}

template <class PairT>
__global__ void __launch_bounds__(kSrcThreads, 1) wsrc_kernel(TravParams p, SrcParams q) {
    extern __shared__ uint32_t s_ring[];  // [2 * R]: queued, then consumed, per slot
    __shared__ int32_t s_ql[64];          // level at which query vertex q settled for this source
    __shared__ double s_dep[64];
    __shared__ double s_msum[64];         // several query vertices: per-column scan sums
    __shared__ unsigned long long s_cd[64];  // ... d(s, croot[c])
    __shared__ double s_red[32];
    __shared__ long long s_i;
    __shared__ int s_k, s_nh, s_err, s_flag, s_stop;
    __shared__ int s_nch[2];  // chunks of the current level, by level parity
    __shared__ unsigned long long s_t0;

    const int tid = threadIdx.x;
    const int bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
    const int R = q.ring;
    const int64_t bcap = q.bcap;
    const int CH = p.chunk_arcs;
    uint32_t *s_cnt = s_ring;
    uint32_t *s_base = s_ring + R;
    const size_t boff = (size_t)blockIdx.x * (size_t)q.n;
    DistSig *ds = q.ds + boff;  // wide pairs (Eq. 4 reads and writes them directly)
    PairT P;
    if constexpr (PairT::kWide)
        P.ds = ds;
    else
        P.w = reinterpret_cast<unsigned long long *>(q.ds) + boff;
    int32_t *hv = q.hv + boff;
    int32_t *lstart = q.lstart + (size_t)blockIdx.x * (size_t)q.maxlev;
    unsigned long long *ldist = q.ldist + (size_t)blockIdx.x * (size_t)q.maxlev;
    uint32_t *bk = q.bk + (size_t)blockIdx.x * (size_t)R * (size_t)bcap;
    Chunk *chs = q.ch + (size_t)blockIdx.x * (size_t)q.chcap;
    double *part = q.part + (size_t)blockIdx.x * (size_t)q.chcap;
    uint32_t *tb = p.mode == kModeSpd ? q.tb + (size_t)blockIdx.x * (size_t)q.tbw : nullptr;
    SrcStats st;
    unsigned long long ns_fwd = 0, ns_bwd = 0, ns_other = 0, t_mark = 0;
    unsigned long long lev_max = 0;
    if (tid == 0) t_mark = global_ns();

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const long long i = (long long)atomicAdd(q.next, 1ull);
            bool stop = i >= q.nsrc || ld_vol(&p.ctr->err) != 0;
            if (!stop && p.cancel && *(volatile const int32_t *)p.cancel != 0) {
                set_err(p.ctr, kDevCancelled);
                stop = true;
            }
            s_i = i;
            s_stop = stop ? 1 : 0;
            s_nh = 0;
            s_err = 0;
            s_flag = 0;
            s_nch[0] = 0;
            s_nch[1] = 0;
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
            s_t0 = t;
        }
        for (int k = tid; k < 2 * R; k += bd) s_ring[k] = 0u;
        for (int k = tid; k < 64; k += bd) {
            s_ql[k] = -1;
            s_dep[k] = 0.0;
            s_msum[k] = 0.0;
        }
        __syncthreads();
        if (s_stop) break;
        const long long si = s_i;
        const int v0 = p.srcs[si];
        if (v0 < 0) continue;
        const uint64_t need = __ldg(p.need + v0);
        if (tid == 0) {
            P.seed(v0);
            bk[0] = (uint32_t)v0;  // slot 0, position 0
            s_cnt[0] = 1u;
        }
        __syncthreads();

        // ---------------- forward: settle distance values in order ----------------
        unsigned long long d = 0;
        int seg = 0, nh = 0;
        bool first = true;
        for (;;) {
            if (tid == 0) s_k = R;
            __syncthreads();
            for (int k = tid + (first ? 0 : 1); k < R; k += bd) {
                const int sl = (int)((d + (unsigned long long)k) & (unsigned long long)(R - 1));
                if (s_cnt[sl] != s_base[sl]) {
                    atomicMin(&s_k, k);
                    break;
                }
            }
            __syncthreads();
            const int kmin = s_k;
            if (kmin >= R) break;
            first = false;
            d += (unsigned long long)kmin;
            const int slot = (int)(d & (unsigned long long)(R - 1));
            const uint32_t b0 = s_base[slot];
            const uint32_t cnt = s_cnt[slot] - b0;
            if (seg + 1 >= q.maxlev || (int64_t)cnt > bcap) {
                if (tid == 0) set_err(p.ctr, seg + 1 >= q.maxlev ? kDevLevelOverflow : kDevBucketOverflow);
                return;
            }
            if (tid == 0) {
                lstart[seg] = nh;
                ldist[seg] = d;
            }
            int *nchp = &s_nch[seg & 1];
            // step 1: the slot's vertices; short rows finish here
            {
                const int lpp = lanes_per_vertex((long long)cnt, bd);
                const int per = 32 / lpp, sub = lane / lpp, rl = lane % lpp;
                const bool lead = rl == 0;
                const long long ngroups = ((long long)cnt + per - 1) / per;
                const uint32_t *bks = bk + (size_t)slot * (size_t)bcap;
                for (long long gi = warp; gi < ngroups; gi += nwarps) {
                    const long long ii = gi * per + sub;
                    int x = 0;
                    unsigned long long xd = PairT::kUnreached;
                    double xs = 0.0;
                    if (ii < (long long)cnt) {
                        x = (int)bks[(b0 + (uint32_t)ii) & (uint32_t)(bcap - 1)];
                        P.get(x, xd, xs);
                    }
                    const bool ok = xd == d;
                    const unsigned am = __ballot_sync(kFull, ok && lead);
                    if (am == 0u) continue;
                    int eb = 0;
                    if (lane == 0) eb = atomicAdd(&s_nh, __popc(am));
                    eb = __shfl_sync(kFull, eb, 0);
                    const int e = eb + __popc(am & ((1u << (sub * lpp)) - 1u));
                    long long rb = 0, re = 0;
                    if (ok) {
                        rb = __ldg(p.off + x);
                        re = __ldg(p.off + x + 1);
                    }
                    if (ok && lead) {
                        hv[e] = x;
                        st.reached += 1;
                        st.edges += (unsigned long long)(re - rb);
                        if (xs >= kSrcTwo53) s_flag = 1;
                        if (*(volatile const int32_t *)(p.tag + x) == -1 && atomicCAS(&p.tag[x], -1, 0) == -1) {
                            st.vb += 1;
                            st.eb += (unsigned long long)(re - rb);
                        }
                        uint64_t y = __ldg(p.qmask + x) & need;
                        while (y) {
                            const int qq = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            s_ql[qq] = seg;
                        }
                    }
                    if (ok && re - rb <= p.wshort) {
                        if (lead) st.arcs += (unsigned long long)(re - rb);
                        const int er = src_relax(p, P, bk, s_cnt, tb, bcap, R, d, xs, rb + rl, re, lpp, st.tight);
                        if (er) {
                            s_err = 1;
                            set_err(p.ctr, er);
                        }
                    } else if (ok && lead) {
                        const int nout = (int)((re - rb + CH - 1) / CH);
                        const int c0 = atomicAdd(nchp, nout);
                        if ((int64_t)c0 + nout > q.chcap) {
                            s_err = 1;
                            set_err(p.ctr, kDevChunkOverflow);
                        } else {
                            src_store_chunks(chs, c0, x, e, 0, rb, re, nout, CH);
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                s_base[slot] = b0 + cnt;
                s_nch[(seg + 1) & 1] = 0;
                if ((double)(global_ns() - s_t0) > p.timeout_ns) {
                    s_err = 1;
                    set_err(p.ctr, kDevTimeout);
                }
            }
            const int nch = *nchp;
            if (s_err) return;
            // step 2: long out-rows, lanes over arcs
            if (nch > 0) {
                for (int c = warp; c < nch; c += nwarps) {
                    const Chunk ch = load_chunk(&chs[c]);
                    unsigned long long cdv;
                    double sg;
                    P.get(ch.v, cdv, sg);
                    const int er = src_relax(p, P, bk, s_cnt, tb, bcap, R, d, sg, ch.a0 + lane, ch.a0 + ch.na, 32, st.tight);
                    if (er) {
                        s_err = 1;
                        set_err(p.ctr, er);
                    }
                    if (lane < ch.na) st.arcs += (unsigned long long)((ch.na - lane + 31) / 32);
                }
                __syncthreads();
                if (s_err) return;
            }
            nh = s_nh;
            ++seg;
        }
        const int nseg = seg;
        if ((unsigned long long)(nseg > 0 ? nseg - 1 : 0) > lev_max) lev_max = (unsigned long long)(nseg > 0 ? nseg - 1 : 0);
        if (tid == 0) {
            const unsigned long long t = global_ns();
            ns_fwd += t - t_mark;
            t_mark = t;
            // the last forward level may have left chunks counted in its slot
            s_nch[0] = 0;
            s_nch[1] = 0;
        }
        __syncthreads();

        if (p.mode == kModeScan && p.ncols < 2) {
            // ---------------- vertex scan, one query vertex r ----------------
            // delta_s.(r) = sigma_sr * sum over settled t with d(r, t) >= 1 and
            // d(s, r) + d(r, t) = d(s, t) of sigma_rt / sigma_st
            const int r = p.vroot;
            unsigned long long dsr;
            double ssr;
            P.get(r, dsr, ssr);
            double acc = 0.0;
            if (dsr != PairT::kUnreached && need) {
                for (int e = tid; e < nh; e += bd) {
                    const int t = hv[e];
                    const unsigned long long rd = p.rdist[t];
                    unsigned long long dt;
                    double sst;
                    P.get(t, dt, sst);
                    if (rd == 0ull || rd >= dt || dsr + rd != dt) continue;
                    acc += p.rsig[t] / sst;
                    st.pairs += 1;
                }
            }
            acc = sum_warp(acc);
            if (lane == 0) s_red[warp] = acc;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int w = 0; w < nwarps; ++w) sum += s_red[w];
                const double dv = dsr != PairT::kUnreached ? ssr * sum : 0.0;
                uint64_t y = need;
                while (y) {
                    const int qq = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    s_dep[qq] = dv;
                }
            }
        } else if (p.mode == kModeScan) {
            // ---------------- vertex scan, several query vertices ----------------
            // column c (query vertex croot[c]) of the queries that need s
            uint64_t cols = 0ull;
            {
                uint64_t y = need;
                while (y) {
                    const int qq = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    cols |= 1ull << p.qcol[qq];
                }
            }
            for (int c = tid; c < 64; c += bd) s_cd[c] = ((cols >> c) & 1ull) ? P.dist(p.croot[c]) : PairT::kUnreached;
            __syncthreads();
            for (int e = tid; e < nh; e += bd) {
                const int t = hv[e];
                unsigned long long dt;
                double sst;
                P.get(t, dt, sst);
                uint64_t y = cols;
                while (y) {
                    const int c = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    const unsigned long long dc = s_cd[c];
                    if (dc == PairT::kUnreached) continue;
                    const unsigned long long rd = p.rdistq[(size_t)t * wcols_stride(p.ncols) + c];
                    if (rd == 0ull || rd >= dt || dc + rd != dt) continue;
                    atomicAdd(&s_msum[c], p.rsigq[(size_t)t * wcols_stride(p.ncols) + c] / sst);
                    st.pairs += 1;
                }
            }
            __syncthreads();
            if (tid == 0) {
                uint64_t y = need;
                while (y) {
                    const int qq = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    const int c = p.qcol[qq];
                    unsigned long long dcr;
                    double scr;
                    P.get(p.croot[c], dcr, scr);
                    s_dep[qq] = s_cd[c] != PairT::kUnreached ? scr * s_msum[c] : 0.0;
                }
            }
        } else if constexpr (PairT::kWide) {
            // ---------------- backward (Eq. 4) over the levels ----------------
            int lstop = 0x7fffffff;
            {
                uint64_t y = need;
                while (y) {
                    const int qq = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    if (s_ql[qq] >= 0 && s_ql[qq] < lstop) lstop = s_ql[qq];
                }
            }
            for (int sg = nseg - 1; sg >= lstop; --sg) {
                const int e0 = lstart[sg];
                const int e1 = sg + 1 < nseg ? lstart[sg + 1] : nh;
                const unsigned long long dk = ldist[sg];
                int *nchp = &s_nch[sg & 1];
                const long long ne = e1 - e0;
                const int lpp = lanes_per_vertex(ne, bd);
                const int per = 32 / lpp, sub = lane / lpp, rl = lane % lpp;
                const bool lead = rl == 0;
                const long long ngroups = (ne + per - 1) / per;
                for (long long gi = warp; gi < ngroups; gi += nwarps) {
                    const long long ii = gi * per + sub;
                    const bool ok = ii < ne;
                    int v = 0;
                    long long rb = 0, re = 0;
                    if (ok) {
                        v = hv[e0 + ii];
                        rb = __ldg(p.off + v);
                        re = __ldg(p.off + v + 1);
                    }
                    const bool shortrow = ok && re - rb <= p.wshort;
                    double acc = 0.0;
                    if (shortrow) acc = src_pull_c(p, ds, tb, dk, rb + rl, re, lpp);
                    acc = sum_lanes(acc, lpp);
                    if (shortrow && lead) {
                        src_finalize(p, ds, need, s_dep, v, acc);
                        st.arcs += (unsigned long long)(re - rb);
                    } else if (ok && !shortrow && lead) {
                        const int nout = (int)((re - rb + CH - 1) / CH);
                        const int c0 = atomicAdd(nchp, nout);
                        if ((int64_t)c0 + nout > q.chcap) {
                            s_err = 1;
                            set_err(p.ctr, kDevChunkOverflow);
                        } else {
                            src_store_chunks(chs, c0, v, (int)(e0 + ii), 0, rb, re, nout, CH);
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    s_nch[(sg + 1) & 1] = 0;
                    if ((double)(global_ns() - s_t0) > p.timeout_ns) {
                        s_err = 1;
                        set_err(p.ctr, kDevTimeout);
                    }
                }
                const int nch = *nchp;
                if (s_err) return;
                if (nch > 0) {
                    for (int c = warp; c < nch; c += nwarps) {
                        const Chunk ch = load_chunk(&chs[c]);
                        const double v = sum_warp(src_pull_c(p, ds, tb, dk, ch.a0 + lane, ch.a0 + ch.na, 32));
                        if (lane == 0) part[c] = v;
                        if (lane < ch.na) st.arcs += (unsigned long long)((ch.na - lane + 31) / 32);
                    }
                    __syncthreads();
                    for (int c = tid; c < nch; c += bd) {
                        const Chunk ch = load_chunk(&chs[c]);
                        if (ch.k == 0) {
                            double acc = 0.0;
                            for (int k = 0; k < ch.nch; ++k) acc += part[c + k];
                            src_finalize(p, ds, need, s_dep, ch.v, acc);
                        }
                    }
                    __syncthreads();
                }
            }
        }
        __syncthreads();
        // ---------------- outputs and reset ----------------
        if (tid < 64 && ((need >> tid) & 1ull)) q.sdep[(size_t)si * 64 + tid] = s_dep[tid];
        if (tid == 0) q.sflag[si] = (uint32_t)s_flag;
        for (int e = tid; e < nh; e += bd) {
            const int x = hv[e];
            P.clear(x);
            if (tb) {
                const long long rb = __ldg(p.off + x), re = __ldg(p.off + x + 1);
                if (re > rb)
                    for (long long w = rb >> 5; w <= (re - 1) >> 5; ++w) tb[w] = 0u;
            }
        }
        if (tid == 0) {
            const unsigned long long t = global_ns();
            ns_bwd += t - t_mark;
            t_mark = t;
        }
    }

    // counters: warp sums, one atomic per warp and counter
    unsigned long long v[7] = {st.edges, st.reached, st.tight, st.arcs, st.vb, st.eb, st.pairs};
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(kFull, v[i], o);
    if (lane == 0) {
        unsigned long long *dst[7] = {&p.ctr->edges, &p.ctr->reached, &p.ctr->tight, &p.ctr->arc_visits,
                                      &p.ctr->vb, &p.ctr->eb, &p.ctr->vpairs};
#pragma unroll
        for (int i = 0; i < 7; ++i)
            if (v[i]) atomicAdd(dst[i], v[i]);
    }
    if (tid == 0) {
        atomicMax(&p.ctr->levels_max, lev_max);
        atomicAdd(&p.ctr->ns_fwd, ns_fwd);
        atomicAdd(&p.ctr->ns_bwd, ns_bwd);
        atomicAdd(&p.ctr->ns_other, ns_other);
    }
}

// Per-tile, per-query sums of the launch's sources (the tile kernel's order:
// eight interleaved partial sums per query, then a fixed shuffle tree), one
// block per tile.
__global__ void wsrc_tile_sums(TravParams p, const double *sdep, const uint32_t *sflag, int S) {
    const long long tile = blockIdx.x;
    const int32_t *tsrc = p.srcs + tile * S;
    for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) {
        const int qq = t >> 3, j = t & 7;
        const bool exact = (p.exact_q >> qq) & 1ull;
        double sum = 0.0;
        int flagged = 0;
        for (int s = j; s < S; s += 8) {
            const int v = tsrc[s];
            if (v < 0) continue;
            double mlt = 0.0;
            if (exact)
                mlt = ((p.need[v] >> qq) & 1ull) ? 1.0 : 0.0;
            else if (p.mult)
                mlt = (double)p.mult[((size_t)tile * S + s) * 64 + qq];
            if (mlt != 0.0) {
                const size_t i = (size_t)tile * S + s;
                sum += mlt * sdep[i * 64 + qq];
                if (sflag[i]) flagged = 1;
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            sum += __shfl_down_sync(kFull, sum, o, 8);
            flagged |= __shfl_down_sync(kFull, flagged, o, 8);
        }
        if (j == 0) {
            p.tile_partial[tile * 64 + qq] = sum;
            if (flagged) atomicOr(&p.qflags[qq], 1u);
        }
    }
}

// Bytes of per-block state for a graph of n vertices.
size_t src_block_bytes(int64_t n, int64_t m, int R, int64_t bcap, int64_t maxlev, int64_t chcap) {
    return (size_t)n * (16 + 4) + (size_t)((m + 31) / 32) * 4 + (size_t)R * (size_t)bcap * 4 + (size_t)maxlev * 12 +
           (size_t)chcap * (32 + 8);
}

// Every vertex unreached: 16-byte pairs (distance all ones, sigma zero) or
// 8-byte words (distance field all ones, count zero).
__global__ void clear_pairs(unsigned long long *ds, size_t nvert, int layout) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvert; i += (size_t)gridDim.x * blockDim.x) {
        if (layout == 1) {
            ds[2 * i] = ~0ull;
            ds[2 * i + 1] = 0ull;  // +0.0
        } else {
            ds[i] = NarrowPairs::kUnreached;
        }
    }
}

// Clears the per-block vertex state in the given layout (1 wide, 2 narrow).
bc_status clear_src_pairs(bc_graph *g, int layout) {
    bcd_workspace &ws = g->ws;
    const size_t nvert = (size_t)ws.sblocks * (size_t)g->n;
    clear_pairs<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(ws.sds, nvert, layout);
    g->launches += 1;
    BCD_CUDA(cudaGetLastError());
    ws.slayout = layout;
    return BC_OK;
}

void free_src_arrays(bcd_workspace &ws) {
    dev_free(ws.sds);
    dev_free(ws.stb);
    dev_free(ws.shv);
    dev_free(ws.slstart);
    dev_free(ws.sldist);
    dev_free(ws.sbk);
    dev_free(ws.sch);
    dev_free(ws.spart);
    ws.sblocks = 0;
}

// (Re)allocates the per-block state for the current capacities; every pair
// starts unreached.
bc_status alloc_src_arrays(bc_graph *g, int blocks) {
    bcd_workspace &ws = g->ws;
    free_src_arrays(ws);
    const size_t B = (size_t)blocks;
    const size_t n = (size_t)g->n;
    BCD_TRY(dev_alloc(&ws.sds, 2 * B * n));
    BCD_TRY(dev_alloc(&ws.stb, B * (size_t)((g->m + 31) / 32)));
    BCD_CUDA(cudaMemsetAsync(ws.stb, 0, sizeof(uint32_t) * B * (size_t)((g->m + 31) / 32), g->stream));
    BCD_TRY(dev_alloc(&ws.shv, B * n));
    BCD_TRY(dev_alloc(&ws.slstart, B * (size_t)ws.smaxlev));
    BCD_TRY(dev_alloc(&ws.sldist, B * (size_t)ws.smaxlev));
    BCD_TRY(dev_alloc(&ws.sbk, B * (size_t)ws.ring * (size_t)ws.sbcap));
    BCD_TRY(dev_alloc(&ws.sch, B * (size_t)ws.schcap));
    BCD_TRY(dev_alloc(&ws.spart, B * (size_t)ws.schcap));
    ws.sblocks = blocks;
    return clear_src_pairs(g, 1);
}

bc_status reset_src_state(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    if (!ws.sds) return BC_OK;
    BCD_TRY(clear_src_pairs(g, ws.slayout ? ws.slayout : 1));
    BCD_CUDA(cudaMemsetAsync(ws.stb, 0, sizeof(uint32_t) * (size_t)ws.sblocks * (size_t)((g->m + 31) / 32), g->stream));
    if (ws.tag) BCD_CUDA(cudaMemsetAsync(ws.tag, 0xff, sizeof(int32_t) * (size_t)g->n, g->stream));
    return BC_OK;
}

template <typename T>
bc_status grow_buf(T **p, int64_t *cap, int64_t need) {
    if (*cap >= need && *p) return BC_OK;
    dev_free(*p);
    *cap = 0;
    const int64_t c = std::max<int64_t>(need, 1024);
    BCD_TRY(dev_alloc(p, (size_t)c));
    *cap = c;
    return BC_OK;
}

}  // namespace

void free_src_state(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    free_src_arrays(ws);
    dev_free(ws.sdep);
    dev_free(ws.sflag);
    dev_free(ws.snext);
    ws.sdep_cap = 0;
    ws.sflag_cap = 0;
    ws.sbcap = 0;
    ws.schcap = 0;
    ws.smaxlev = 0;
    ws.slayout = 0;
    ws.swide = false;
}

bool src_kernel_applies(const bc_graph *g, const TravParams &p) {
    return g->weighted && g->weighted_kernel == 2 && (p.mode == kModeSpd || p.mode == kModeScan) &&
           !(p.flags & (kFlagNoBackward | kFlagNoReset | kFlagFullBackward | kFlagRootOut));
}

bc_status run_src_traversal(bc_graph *g, int W, TravParams &p, int *levels_out, unsigned long long *edges_out) {
    bcd_workspace &ws = g->ws;
    BCD_TRY(ensure_weighted_state(g));  // ring size, tag array
    const int threads = kSrcThreads;
    const int S = 64 * W;
    const int64_t nsrc = p.ntiles * S;
    const int R = ws.ring;
    const size_t smem = sizeof(uint32_t) * 2 * (size_t)R;
    int per_sm = 0, per_sm_n = 0;
    BCD_CUDA(cudaFuncSetAttribute(wsrc_kernel<WidePairs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BCD_CUDA(cudaFuncSetAttribute(wsrc_kernel<NarrowPairs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wsrc_kernel<WidePairs>, threads, smem));
    BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_n, wsrc_kernel<NarrowPairs>, threads, smem));
    per_sm = std::min(per_sm, per_sm_n);
    if (per_sm < 1) return set_error(BC_E_INTERNAL, "weighted source kernel cannot be resident");
    if (ws.sbcap == 0) {
        // queued vertices of one distance of one source: a few times the
        // average vertices per distance value, and at least 2^21 entries
        // over the whole ring (8 MB); grown on overflow
        int64_t b = 64;
        while ((b < 4 * (int64_t)g->n / R || b * R < ((int64_t)1 << 21)) && b < ((int64_t)1 << 30)) b *= 2;
        ws.sbcap = b;
        ws.schcap = 16384;
        ws.smaxlev = 8192;
    }
    int blocks = g->num_sms * per_sm;
    {
        size_t fr = 0, tot = 0;
        BCD_CUDA(cudaMemGetInfo(&fr, &tot));
        const size_t have = ws.sblocks > 0 ? src_block_bytes(g->n, g->m, R, ws.sbcap, ws.smaxlev, ws.schcap) * ws.sblocks : 0;
        const size_t per = src_block_bytes(g->n, g->m, R, ws.sbcap, ws.smaxlev, ws.schcap);
        const size_t budget = (fr + have) / 2;
        blocks = (int)std::min<size_t>((size_t)blocks, budget / per);
        if (blocks < 1) return set_error(BC_E_OOM, "weighted source kernel: no room for one block's state");
    }
    if (ws.sblocks != blocks || !ws.sds) {
        const bc_status st = alloc_src_arrays(g, blocks);
        if (st != BC_OK) {
            free_src_arrays(ws);
            return st;
        }
    }
    BCD_TRY(grow_buf(&ws.sdep, &ws.sdep_cap, nsrc * 64));
    BCD_TRY(grow_buf(&ws.sflag, &ws.sflag_cap, nsrc));
    if (!ws.snext) BCD_TRY(dev_alloc(&ws.snext, 1));
    for (int attempt = 0; attempt < 8; ++attempt) {
        p.off = g->d_off;
        p.col = g->d_col;
        p.wt = g->d_w;
        p.roff = g->d_roff;
        p.rcol = g->d_rcol;
        p.rwt = g->d_rw;
        p.tag = ws.tag;
        p.ctr = ws.ctr;
        p.n = g->n;
        p.chunk_arcs = g->chunk_arcs;
        p.wshort = g->wshort;
        p.timeout_ns = g->timeout_ns;
        p.cancel = g->cancel_d;
        SrcParams q;
        q.ds = reinterpret_cast<DistSig *>(ws.sds);
        q.hv = ws.shv;
        q.lstart = ws.slstart;
        q.ldist = ws.sldist;
        q.bk = ws.sbk;
        q.ch = ws.sch;
        q.part = ws.spart;
        q.tb = ws.stb;
        q.tbw = (g->m + 31) / 32;
        q.sdep = ws.sdep;
        q.sflag = ws.sflag;
        q.next = ws.snext;
        q.n = g->n;
        q.bcap = ws.sbcap;
        q.chcap = ws.schcap;
        q.nsrc = nsrc;
        q.ring = R;
        q.maxlev = ws.smaxlev;
        // 8-byte words for vertex-scan launches, unless one of this graph
        // has overflowed them; the Eq. 4 pass needs the 16-byte pairs
        const int layout = (p.mode == kModeScan && !ws.swide) ? 2 : 1;
        if (ws.slayout != layout) BCD_TRY(clear_src_pairs(g, layout));
        BCD_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), g->stream));
        BCD_CUDA(cudaMemsetAsync(ws.snext, 0, sizeof(unsigned long long), g->stream));
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        const bool timed = cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess;
        if (timed) cudaEventRecord(ev0, g->stream);
        if (layout == 2)
            wsrc_kernel<NarrowPairs><<<(unsigned)ws.sblocks, (unsigned)threads, smem, g->stream>>>(p, q);
        else
            wsrc_kernel<WidePairs><<<(unsigned)ws.sblocks, (unsigned)threads, smem, g->stream>>>(p, q);
        g->launches += 1;
        g->last_grid = ws.sblocks;
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            if (timed) {
                cudaEventDestroy(ev0);
                cudaEventDestroy(ev1);
            }
            return cuda_error(le, "wsrc_kernel launch");
        }
        if (timed) cudaEventRecord(ev1, g->stream);
        Counters c;
        BCD_CUDA(cudaMemcpyAsync(&c, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, g->stream));
        BCD_CUDA(cudaStreamSynchronize(g->stream));
        float ms = 0.f;
        if (timed) {
            cudaEventElapsedTime(&ms, ev0, ev1);
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
        }
        // the tag array marks the launch's union of reached vertices; clear it
        BCD_CUDA(cudaMemsetAsync(ws.tag, 0xff, sizeof(int32_t) * (size_t)g->n, g->stream));
        if (c.err == kDevOk) {
            if (p.ntiles > 0) {
                wsrc_tile_sums<<<(unsigned)p.ntiles, 512, 0, g->stream>>>(p, ws.sdep, ws.sflag, S);
                g->launches += 1;
                BCD_CUDA(cudaGetLastError());
            }
            g->last = c;
            g->last_ms_launch = ms;
            // phase times: the blocks' summed phase times, scaled to the launch
            const double tot = (double)c.ns_fwd + (double)c.ns_bwd + (double)c.ns_other;
            const double launch_ns = (double)ms * 1e6;
            g->last_ns_fwd = tot > 0 ? (unsigned long long)(launch_ns * (double)c.ns_fwd / tot) : 0ull;
            g->last_ns_bwd = tot > 0 ? (unsigned long long)(launch_ns * (double)c.ns_bwd / tot) : 0ull;
            g->last_ns_other = tot > 0 ? (unsigned long long)(launch_ns * (double)c.ns_other / tot) : 0ull;
            if (levels_out) *levels_out = (int)c.levels_max;
            if (edges_out) *edges_out = c.edges;
            return BC_OK;
        }
        BCD_TRY(reset_src_state(g));
        if (p.qflags) BCD_CUDA(cudaMemsetAsync(p.qflags, 0, sizeof(uint32_t) * 64, g->stream));
        if (c.err == kDevTimeout) return set_error(BC_E_TIMEOUT, "weighted source kernel: a source ran past the time limit");
        if (c.err == kDevCancelled) return set_error(BC_E_CANCELLED, "traversal: cancelled by bc_cancel");
        if (c.err == kDevWide) {
            // a count of 2^40 or a distance of 2^24 - 1: 16-byte pairs from now on
            ws.swide = true;
            continue;
        }
        const size_t before = (size_t)ws.sblocks * src_block_bytes(g->n, g->m, R, ws.sbcap, ws.smaxlev, ws.schcap);
        if (c.err == kDevBucketOverflow) {
            if (ws.sbcap >= ((int64_t)1 << 30)) return set_error(BC_E_OOM, "bucket ring: too many queued vertices at one distance");
            ws.sbcap *= 2;
        } else if (c.err == kDevLevelOverflow) {
            if (ws.smaxlev >= (1 << 28)) return set_error(BC_E_OOM, "traversal: more distance levels than the arrays hold");
            ws.smaxlev *= 4;
        } else if (c.err == kDevChunkOverflow) {
            if (ws.schcap >= ((int64_t)1 << 30)) return set_error(BC_E_OOM, "traversal: too many long-row chunks in one level");
            ws.schcap *= 4;
        } else {
            return set_error(BC_E_INTERNAL, "weighted source kernel: unexpected device error");
        }
        // grow, within half of the memory free besides the current state
        size_t fr = 0, tot = 0;
        BCD_CUDA(cudaMemGetInfo(&fr, &tot));
        const size_t per = src_block_bytes(g->n, g->m, R, ws.sbcap, ws.smaxlev, ws.schcap);
        const int nb = (int)std::min<size_t>((size_t)ws.sblocks, ((fr + before) / 2) / per);
        if (nb < 1) {
            free_src_arrays(ws);
            return set_error(BC_E_OOM, "weighted source kernel: no room for one block's state");
        }
        const bc_status st = alloc_src_arrays(g, nb);
        if (st != BC_OK) {
            free_src_arrays(ws);
            return st;
        }
    }
    return set_error(BC_E_OOM, "weighted source kernel: state did not fit after growing it");
}

}  // namespace bcd
