// Persistent multi-source traversal: the single-source work of Algorithm 1
// (and Algorithm 2) for S = 64*W sources at once.
//
// One cooperative launch walks every tile of S sources. Per tile:
//   forward  (Section 2): level-synchronous BFS over the forward CSR, one
//            grid barrier per level. Per vertex the dense state holds the
//            visited mask and two level-parity masks (bit s: vertex is at the
//            current / next level for source s). Frontier vertices are pushed
//            along their out-arcs in chunks of at most chunk_arcs arcs; for
//            every arc (u, v) the sources newly reaching v are
//            F(u) & ~(visited(v) | current(v)), and sigma_s(v) += sigma_s(u)
//            by an fp64 atomic add (sigma are integers, so the sum is exact
//            in any order while below 2^53).
//   backward (Eq. 4): levels from the deepest one up to the shallowest level
//            any query vertex sits at. With c_s(w) = (1 + delta_s(w)) /
//            sigma_s(w), delta_s(v) = sigma_s(v) * sum over tight out-arcs
//            (v, w) of c_s(w). The sum is pushed: the entries of level L + 1
//            add c_s(w) along their tight in-arcs (R(G), in chunks) into an
//            accumulator slab acc[v][s] with fp64 atomic adds, which do not
//            hold the warp; after a barrier the level-L entries turn acc
//            into delta and c. The sum order follows the schedule, so delta
//            can differ from run to run in its last bits.
// Scan mode (every query of the launch at one vertex r) keeps the forward
//            pass and replaces the backward by one pass over the reached
//            (vertex, source) pairs: delta_s.(r) = sigma_sr * sum of
//            sigma_rt / sigma_st over the t behind r on a shortest s-t path,
//            with d(r, t) and sigma_rt from an earlier scan-mode launch whose
//            only source is r (kFlagRootOut).
// Reach mode (RV(r), Section 4.1) runs the forward pass only, over R(G),
// with one source slot per query root, and ORs every level mask into rvmask.
//
// Every grid barrier wait is bounded; a timeout or a capacity overflow sets
// Counters::err and all blocks leave.
#include <cooperative_groups.h>

#include <algorithm>

#include "bcd_common.cuh"
#include "bcd_device.cuh"

namespace bcd {

namespace {

using namespace dev;

// Appends the vertices a warp discovered at level L+1: one entry and its
// out-arc chunks each and, in SPD mode, the in-arc (R(G)) chunks the backward
// pass pushes along, with one set of counter atomics per warp.
template <int W, int MODE>
__device__ __forceinline__ void warp_append(const TravParams &p, int L, bool app, int wv, int wnch, long long wrb,
                                            long long wre, int winch, long long wirb, long long wire, long long es1,
                                            long long cs1, long long ics1, int lane) {
    const unsigned am = __ballot_sync(kFull, app);
    if (am == 0) return;
    const int rank = __popc(am & ((1u << lane) - 1u));
    const int ne = __popc(am);
    int x = app ? wnch : 0;
    int xi = app ? winch : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        const int yi = __shfl_up_sync(kFull, xi, o);
        if (lane >= o) {
            x += y;
            xi += yi;
        }
    }
    const int tot = __shfl_sync(kFull, x, 31);
    const int toti = __shfl_sync(kFull, xi, 31);
    // out-arcs of the appended vertices: the next level's frontier arcs, which
    // choose its direction
    unsigned long long fa = app ? (unsigned long long)(wre - wrb) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fa += __shfl_xor_sync(kFull, fa, o);
    unsigned long long eb = 0, cb = 0, ib = 0;
    if (lane == 0) {
        // entries (low half) and out-arc chunks (high half) in one atomic: every
        // appending warp of the level meets on this word
        const unsigned long long old =
            atomicAdd(&p.lev_grab[4 * ((long long)p.maxlev + 2) + L + 1], (unsigned long long)ne | ((unsigned long long)tot << 32));
        eb = old & 0xffffffffull;
        cb = old >> 32;
        if (MODE == kModeSpd && toti)
            ib = atomicAdd(&p.lev_grab[2 * ((long long)p.maxlev + 2) + L + 1], (unsigned long long)toti);
        if (MODE != kModeReach && fa && p.pull_arcs_min > 0)
            atomicAdd(&p.lev_grab[3 * ((long long)p.maxlev + 2) + L + 1], fa);
    }
    eb = __shfl_sync(kFull, eb, 0);
    cb = __shfl_sync(kFull, cb, 0);
    if (MODE == kModeSpd) ib = __shfl_sync(kFull, ib, 0);
    if (app) {
        const long long e = es1 + (long long)eb + rank;
        const long long c0 = cs1 + (long long)cb + (x - wnch);
        const long long i0 = ics1 + (long long)ib + (xi - winch);
        if (e >= p.hcap) {
            set_err(p.ctr, kDevHistOverflow);
        } else if (c0 + wnch > p.ccap || (MODE == kModeSpd && i0 + winch > p.ccap)) {
            set_err(p.ctr, kDevChunkOverflow);
        } else {
            p.hv[e] = wv;
            emit_chunks(p, c0, wv, (int)e, wnch, wrb, wre);
            if (MODE == kModeSpd) {
                const int CH = p.chunk_arcs;
                for (int k = 0; k < winch; ++k) {
                    const long long a0 = wirb + (long long)k * CH;
                    store_chunk(&p.ichunks[i0 + k], wv, (int)e, k, winch, a0, (int)(min(wire, a0 + CH) - a0));
                }
            }
        }
    }
}

// Level 0 of a tile: one entry per source slot (block 0 only). Thread t
// seeds slot t: the launch has at least S threads per block.
template <int W, int MODE>
__device__ void init_tile(const TravParams &p, const int32_t *tsrc) {
    constexpr int S = 64 * W;
    __shared__ int s_scan[S];
    __shared__ int s_valid;
    const int t = threadIdx.x;
    int v = -1, nch = 0;
    long long rb = 0, re = 0;
    if (t < S) {
        v = tsrc[t];
        if (v >= 0) {
            rb = p.off[v];
            re = p.off[v + 1];
            nch = (int)max(1ll, (re - rb + p.chunk_arcs - 1) / p.chunk_arcs);
        }
        s_scan[t] = nch;
    }
    if (t == 0) s_valid = 0;
    __syncthreads();
    if (t < S && v >= 0) atomicAdd(&s_valid, 1);
    for (int o = 1; o < S; o <<= 1) {
        int y = 0;
        if (t < S && t >= o) y = s_scan[t - o];
        __syncthreads();
        if (t < S) s_scan[t] += y;
        __syncthreads();
    }
    if (t < S && v >= 0) {
        const int c0 = s_scan[t] - nch;
        if (c0 + nch > p.ccap || t >= p.hcap) {
            set_err(p.ctr, kDevChunkOverflow);
        } else {
            uint64_t *row = p.vs + (size_t)v * p.vs_stride;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t b = (w == (t >> 6)) ? (1ull << (t & 63)) : 0ull;
                p.hm[(size_t)t * W + w] = b;
                row[W + w] = b;  // level-0 parity mask
            }
            p.hv[t] = v;
            p.tag[v] = 0;
            emit_chunks(p, c0, v, t, nch, rb, re);
            if (MODE != kModeReach) {
                atomicAdd(&p.ctr->vb, 1ull);
                atomicAdd(&p.ctr->eb, (unsigned long long)(re - rb));
            }
            if (MODE != kModeReach) p.sigma[(size_t)v * S + t] = 1.0;
        }
    }
    if (MODE != kModeReach) {
        for (int i = t; i < S * 64; i += blockDim.x) p.qlevel[i] = -1;
        if (t < W) p.srcflag[t] = 0ull;
    }
    if (MODE == kModeScan && t < S) p.vsum[t] = 0.0;
    if (MODE == kModeScan && p.ncols >= 2)
        for (int i = t; i < S * 64; i += blockDim.x) p.msum[i] = 0.0;
    __syncthreads();
    if (t == 0) {
        p.lev_cnt[0] = (unsigned long long)s_valid;
        p.lev_ccnt[0] = (unsigned long long)s_scan[S - 1];
        p.lev_grab[4 * ((long long)p.maxlev + 2)] = (unsigned long long)s_valid | ((unsigned long long)s_scan[S - 1] << 32);
    }
}

// Expansion of level L (forward pass, Section 2 / Section 4.1). Lane l holds
// sources l + 32 i; the next 32 heads are fetched while the current ones'
// masks are read.
// Per-thread work counters (32-bit; flushed to the 64-bit launch totals at
// the end of every tile).
struct Stats {
    unsigned edges = 0, reached = 0, tight = 0, arcs = 0, vb = 0, eb = 0;
};

__device__ __forceinline__ void flush_stats(Counters *c, Stats &st, int lane) {
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
    st = Stats();
}

// Expansion of one out-arc chunk of a level-L entry (forward pass): the
// descriptor, the frontier mask F of its vertex and this lane's first head
// come in loaded, so the caller can fetch them ahead of time.
template <int W, int MODE>
__device__ __forceinline__ void expand_chunk(const TravParams &p, int L, const Chunk &ch, const uint64_t (&F)[W],
                                             int wv_next, long long es1, long long cs1, long long ics1, Stats &st,
                                             const uint64_t *s_need) {
    constexpr int S = 64 * W;
    constexpr int PL = 2 * W;
    const int lane = threadIdx.x & 31;
    const int cur = 1 + (L & 1);
    const int nxt = 1 + ((L + 1) & 1);
    const int stride = p.vs_stride;
    const int CH = p.chunk_arcs;
    const int v = ch.v, e = ch.e;
    const long long a0 = ch.a0;
    const int na = ch.na;
    double sig[PL];
    if (MODE != kModeReach) {
        // only the frontier's sources: sectors of the row without one are not read
#pragma unroll
        for (int ii = 0; ii < PL; ++ii)
            sig[ii] = mask_bit<W>(F, lane + 32 * ii) ? p.sigma[(size_t)v * S + lane + 32 * ii] : 0.0;
    }
    if (ch.k == 0) {
        if (MODE == kModeReach && p.levout && lane == 0 && p.levout[v] < 0) p.levout[v] = L;
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (lane == w) p.hm[(size_t)e * W + w] = F[w];
        // visited |= F: reductions that need no answer (the sources of F are
        // already excluded from new bits by the current-level mask)
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (lane == w) atomicOr((unsigned long long *)&p.vs[(size_t)v * stride + w], (unsigned long long)F[w]);
        if (MODE != kModeReach) {
            if (lane == 0) {
                int pc = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) pc += __popcll(F[w]);
                st.edges += (unsigned)pc * (unsigned)ch.pad;  // out-degree of v rides in the chunk
                st.reached += (unsigned)pc;
            }
            const uint64_t qm = p.qmask[v];
#pragma unroll
            for (int ii = 0; ii < PL; ++ii) {
                const int s = lane + 32 * ii;
                if (mask_bit<W>(F, s)) {
                    if (qm) {
                        uint64_t x = qm & s_need[s];
                        while (x) {
                            const int q = __ffsll((long long)x) - 1;
                            x &= x - 1;
                            p.qlevel[s * 64 + q] = L;
                        }
                    }
                    if (sig[ii] >= 9007199254740992.0)
                        atomicOr((unsigned long long *)&p.srcflag[s >> 6], 1ull << (s & 63));
                }
            }
        }
    }
    for (int base = 0; base < na; base += 32) {
        const bool valid = base + lane < na;
        const int wv = wv_next;
        wv_next = base + 32 + lane < na ? p.col[a0 + base + 32 + lane] : 0;
        uint64_t nm[W];
        bool any = false;
        if (valid) {
            const uint64_t *wrow = p.vs + (size_t)wv * stride;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                nm[w] = F[w] & ~(wrow[w] | wrow[cur * W + w]);
                any |= nm[w] != 0ull;
            }
            if (MODE != kModeReach) {
                st.arcs += 1;
#pragma unroll
                for (int w = 0; w < W; ++w) st.tight += (unsigned)__popcll(nm[w]);
            }
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) nm[w] = 0ull;
        }
        // heads with new sources: mark them for the next level and claim
        // the level's entry; the claim's answer (and the row bounds) are
        // used only after the sigma adds, so their round trips overlap
        int old = 0x7fffffff;
        long long wrb = 0, wre = 0, wirb = 0, wire = 0;
        if (any) {
            uint64_t *wrow = p.vs + (size_t)wv * stride;
#pragma unroll
            for (int w = 0; w < W; ++w)
                if (nm[w]) atomicOr((unsigned long long *)&wrow[nxt * W + w], (unsigned long long)nm[w]);
            old = atomicMax(&p.tag[wv], L + 1);
            wrb = p.off[wv];
            wre = p.off[wv + 1];
            if (MODE == kModeSpd) {
                wirb = p.roff[wv];
                wire = p.roff[wv + 1];
            }
        }
        if (MODE != kModeReach) {
            // two tight heads per step: their shuffles and atomics overlap
            unsigned bal = __ballot_sync(kFull, any);
            while (bal) {
                const int i0 = __ffs(bal) - 1;
                bal &= bal - 1;
                const int i1 = bal ? __ffs(bal) - 1 : -1;
                if (bal) bal &= bal - 1;
                const int j1 = i1 < 0 ? i0 : i1;
                const int w0 = __shfl_sync(kFull, wv, i0);
                const int w1 = __shfl_sync(kFull, wv, j1);
                uint64_t n0[W], n1[W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    n0[w] = __shfl_sync(kFull, nm[w], i0);
                    n1[w] = __shfl_sync(kFull, nm[w], j1);
                }
                if (i1 < 0) {
#pragma unroll
                    for (int w = 0; w < W; ++w) n1[w] = 0ull;
                }
                double *r0 = p.sigma + (size_t)w0 * S;
                double *r1 = p.sigma + (size_t)w1 * S;
#pragma unroll
                for (int ii = 0; ii < PL; ++ii) {
                    const int s = lane + 32 * ii;
                    if (mask_bit<W>(n0, s)) atomicAdd(&r0[s], sig[ii]);
                    if (mask_bit<W>(n1, s)) atomicAdd(&r1[s], sig[ii]);
                }
            }
        }
        const bool app = any && old < L + 1;
        int wnch = 0, winch = 0;
        if (app) {
            wnch = (int)max(1ll, (wre - wrb + CH - 1) / CH);
            if (MODE == kModeSpd) winch = (int)((wire - wirb + CH - 1) / CH);
            if (MODE != kModeReach && old < 0) {
                st.vb += 1;
                st.eb += (unsigned)(wre - wrb);
            }
        }
        warp_append<W, MODE>(p, L, app, wv, wnch, wrb, wre, winch, wirb, wire, es1, cs1, ics1, lane);
    }
}

// Expansion of level L (forward pass, Section 2 / Section 4.1). A warp takes
// the level's chunks from the dynamic hand-out. With PIPE (the one-block-per-
// SM kernels, which have the registers) the loop runs three chunks deep: the
// descriptor of chunk i + 2 and the frontier mask and first heads of chunk
// i + 1 are in flight while chunk i expands, so a chunk starts with one round
// trip (sigma and the heads' masks) instead of three.
template <int W, int MODE, bool PIPE>
__device__ void forward_level(const TravParams &p, int L, long long cs, long long ccnt, long long es1,
                              long long cs1, long long ics1, Stats &st, const uint64_t *s_need,
                              long long gwarp, long long nwarps) {
    const int lane = threadIdx.x & 31;
    const int cur = 1 + (L & 1);
    const int stride = p.vs_stride;
    ChunkGrabber grab(&p.lev_grab[L], ccnt, nwarps);
    if (!PIPE) {
        long long c;
        while (grab.next(c, lane)) {
            const Chunk ch = load_chunk(&p.chunks[cs + c]);
            const int w0 = lane < ch.na ? p.col[ch.a0 + lane] : 0;
            const uint64_t *vrow = p.vs + (size_t)ch.v * stride;
            uint64_t F[W];
#pragma unroll
            for (int w = 0; w < W; ++w) F[w] = vrow[cur * W + w];
            expand_chunk<W, MODE>(p, L, ch, F, w0, es1, cs1, ics1, st, s_need);
        }
        return;
    }
    Chunk d0{}, d1{};
    long long c0 = 0, c1 = 0;
    bool h0 = grab.next(c0, lane);
    if (h0) d0 = load_chunk(&p.chunks[cs + c0]);
    bool h1 = h0 && grab.next(c1, lane);
    if (h1) d1 = load_chunk(&p.chunks[cs + c1]);
    uint64_t F0[W];
    int w0 = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) F0[w] = 0ull;
    if (h0) {
        const uint64_t *vrow = p.vs + (size_t)d0.v * stride;
#pragma unroll
        for (int w = 0; w < W; ++w) F0[w] = vrow[cur * W + w];
        w0 = lane < d0.na ? p.col[d0.a0 + lane] : 0;
    }
    while (h0) {
        // chunk i + 2: descriptor; chunk i + 1: frontier mask and first heads
        Chunk d2{};
        long long c2 = 0;
        const bool h2 = h1 && grab.next(c2, lane);
        if (h2) d2 = load_chunk(&p.chunks[cs + c2]);
        uint64_t F1[W];
        int w1 = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) F1[w] = 0ull;
        if (h1) {
            const uint64_t *vrow = p.vs + (size_t)d1.v * stride;
#pragma unroll
            for (int w = 0; w < W; ++w) F1[w] = vrow[cur * W + w];
            w1 = lane < d1.na ? p.col[d1.a0 + lane] : 0;
        }
        expand_chunk<W, MODE>(p, L, d0, F0, w0, es1, cs1, ics1, st, s_need);
        h0 = h1;
        d0 = d1;
#pragma unroll
        for (int w = 0; w < W; ++w) F0[w] = F1[w];
        w0 = w1;
        h1 = h2;
        d1 = d2;
    }
}

// Bottom-up step of level L (the forward pass of Section 2 read from the
// other end): sigma_s(v) is the sum of sigma_s(u) over the in-neighbours u
// of v at level L for s, so every vertex v that some source of the tile has
// not reached yet (U = valid & ~(visited(v) | current(v))) scans its in-arcs
// in R(G), and for each in-neighbour u the sources of current(u) & U reach v
// at level L + 1, each adding sigma_s(u). The sums stay in registers: a
// vertex whose in-arcs fit one chunk writes its sigma row and its next-level
// mask once, with no atomic per arc (longer rows are cut into chunks that
// meet in fp64 atomic adds, exact for integers below 2^53). Lane l holds
// sources l + 32 i, as in the push. The level-L entries themselves get the
// bookkeeping the push does for the first chunk of an entry: masks into the
// history, visited |= F, work counters, query levels and the 2^53 check.
// Appends are gathered in a per-warp buffer (lane i holds the i-th) and go
// out 32 at a time through warp_append.
template <int W, int MODE>
__device__ __noinline__ void pull_level(const TravParams &p, int L, long long es, long long es1, long long cs1, long long ics1,
                           Stats &st, const uint64_t *s_need, const uint64_t *s_valid, long long gwarp,
                           long long nwarps) {
    constexpr int S = 64 * W;
    constexpr int PL = 2 * W;
    const int lane = threadIdx.x & 31;
    const int cur = 1 + (L & 1);
    const int nxt = 1 + ((L + 1) & 1);
    const int stride = p.vs_stride;
    const int CH = p.chunk_arcs;
    // (1) the level-L entries, one warp each
    for (long long e = es + gwarp; e < es1; e += nwarps) {
        const int v = p.hv[e];
        const uint64_t *vrow = p.vs + (size_t)v * stride;
        uint64_t F[W];
#pragma unroll
        for (int w = 0; w < W; ++w) F[w] = vrow[cur * W + w];
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (lane == w) {
                p.hm[(size_t)e * W + w] = F[w];
                atomicOr((unsigned long long *)&p.vs[(size_t)v * stride + w], (unsigned long long)F[w]);
            }
        if (lane == 0) {
            int pc = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) pc += __popcll(F[w]);
            st.edges += (unsigned)pc * (unsigned)(p.off[v + 1] - p.off[v]);
            st.reached += (unsigned)pc;
        }
        const uint64_t qm = p.qmask[v];
        const double *srow = p.sigma + (size_t)v * S;
#pragma unroll
        for (int ii = 0; ii < PL; ++ii) {
            const int s = lane + 32 * ii;
            if (mask_bit<W>(F, s)) {
                if (qm) {
                    uint64_t x = qm & s_need[s];
                    while (x) {
                        const int q = __ffsll((long long)x) - 1;
                        x &= x - 1;
                        p.qlevel[s * 64 + q] = L;
                    }
                }
                if (srow[s] >= 9007199254740992.0)
                    atomicOr((unsigned long long *)&p.srcflag[s >> 6], 1ull << (s & 63));
            }
        }
    }
    // (2) every vertex's in-arc chunks, handed out dynamically
    int bv = 0, bnch = 0, binch = 0, bcnt = 0;
    long long brb = 0, bre = 0, birb = 0, bire = 0;
    ChunkGrabber grab(&p.lev_grab[L], p.npchunks, nwarps);
    long long c;
    while (grab.next(c, lane)) {
        const int2 pc = p.pchunks[c];
        const int v = pc.x;
        const uint64_t *vrow = p.vs + (size_t)v * stride;
        uint64_t U[W];
        bool anyu = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            U[w] = s_valid[w] & ~(vrow[w] | vrow[cur * W + w]);
            anyu |= U[w] != 0ull;
        }
        if (!anyu) continue;  // every source of the tile has reached v
        const long long rb = p.roff[v], re = p.roff[v + 1];
        const long long a0 = rb + (long long)pc.y * CH;
        const int na = (int)min((long long)CH, re - a0);
        const int nch = (int)((re - rb + CH - 1) / CH);
        double acc[PL];
#pragma unroll
        for (int ii = 0; ii < PL; ++ii) acc[ii] = 0.0;
        unsigned lm = 0;  // bit ii: source lane + 32 ii reaches v here
        int unext = lane < na ? p.rcol[a0 + lane] : 0;
        for (int base = 0; base < na; base += 32) {
            const bool valid = base + lane < na;
            const int u = unext;
            unext = base + 32 + lane < na ? p.rcol[a0 + base + 32 + lane] : 0;
            uint64_t t[W];
            bool any = false;
            if (valid) {
                const uint64_t *urow = p.vs + (size_t)u * stride;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    t[w] = urow[cur * W + w] & U[w];
                    any |= t[w] != 0ull;
                }
                st.arcs += 1;
#pragma unroll
                for (int w = 0; w < W; ++w) st.tight += (unsigned)__popcll(t[w]);
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w) t[w] = 0ull;
            }
            // two tight in-neighbours per step: their gathers overlap
            unsigned bal = __ballot_sync(kFull, any);
            while (bal) {
                const int i0 = __ffs(bal) - 1;
                bal &= bal - 1;
                const int i1 = bal ? __ffs(bal) - 1 : -1;
                if (bal) bal &= bal - 1;
                const int j1 = i1 < 0 ? i0 : i1;
                const int u0 = __shfl_sync(kFull, u, i0);
                const int u1 = __shfl_sync(kFull, u, j1);
                uint64_t n0[W], n1[W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    n0[w] = __shfl_sync(kFull, t[w], i0);
                    n1[w] = i1 < 0 ? 0ull : __shfl_sync(kFull, t[w], j1);
                }
                const double *r0 = p.sigma + (size_t)u0 * S;
                const double *r1 = p.sigma + (size_t)u1 * S;
#pragma unroll
                for (int ii = 0; ii < PL; ++ii) {
                    const int s = lane + 32 * ii;
                    const bool b0 = mask_bit<W>(n0, s), b1 = mask_bit<W>(n1, s);
                    const double x0 = b0 ? r0[s] : 0.0;
                    const double x1 = b1 ? r1[s] : 0.0;
                    acc[ii] += x0 + x1;
                    if (b0 | b1) lm |= 1u << ii;
                }
            }
        }
        uint64_t nm[W];
        bool anynm = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const unsigned lo = __ballot_sync(kFull, (lm >> (2 * w)) & 1u);
            const unsigned hi = __ballot_sync(kFull, (lm >> (2 * w + 1)) & 1u);
            nm[w] = (uint64_t)lo | ((uint64_t)hi << 32);
            anynm |= nm[w] != 0ull;
        }
        if (!anynm) continue;
        // the next-level mask (atomic: the stale level L - 1 bits of this slot
        // are being cleared at the same time) and sigma
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (lane == w && nm[w])
                atomicOr((unsigned long long *)&p.vs[(size_t)v * stride + nxt * W + w], (unsigned long long)nm[w]);
        double *srow = p.sigma + (size_t)v * S;
#pragma unroll
        for (int ii = 0; ii < PL; ++ii)
            if ((lm >> ii) & 1u) {
                if (nch == 1)
                    srow[lane + 32 * ii] = acc[ii];
                else
                    atomicAdd(&srow[lane + 32 * ii], acc[ii]);
            }
        int old = 0;
        if (lane == 0) old = atomicMax(&p.tag[v], L + 1);
        old = __shfl_sync(kFull, old, 0);
        if (old < L + 1) {
            const long long wrb = p.off[v], wre = p.off[v + 1];
            if (lane == 0 && old < 0) {
                st.vb += 1;
                st.eb += (unsigned)(wre - wrb);
            }
            if (lane == bcnt) {
                bv = v;
                brb = wrb;
                bre = wre;
                bnch = (int)max(1ll, (wre - wrb + CH - 1) / CH);
                birb = rb;
                bire = re;
                binch = MODE == kModeSpd ? nch : 0;
            }
            if (++bcnt == 32) {
                warp_append<W, MODE>(p, L, true, bv, bnch, brb, bre, binch, birb, bire, es1, cs1, ics1, lane);
                bcnt = 0;
            }
        }
    }
    warp_append<W, MODE>(p, L, lane < bcnt, bv, bnch, brb, bre, binch, birb, bire, es1, cs1, ics1, lane);
}

// Eq. 4, push form, from level L into level L - 1: each entry w of level L
// sends c_s(w) = (1 + delta_s(w)) / sigma_s(w), with delta_s(w) =
// sigma_s(w) * acc_s(w) complete (level L + 1 pushed into it in the previous
// step), back along its in-arcs (v, w) that are tight for a source s still
// active at L - 1 (v at level L - 1 for s), adding it to acc_s(v) with fp64
// atomic adds. c is formed on the fly from the sigma and acc slabs, which this
// step only reads for level-L pairs. The in-arc chunks of level L were cut in
// the forward pass. Lane l holds sources l + 32 i; two tight tails per step.
template <int W>
__device__ void push_level(const TravParams &p, int L, long long ics, long long ccnt, const uint64_t *s_act,
                           long long nwarps, Stats &st) {
    constexpr int S = 64 * W;
    constexpr int PL = 2 * W;
    const int lane = threadIdx.x & 31;
    const int par = 1 + ((L - 1) & 1);  // parity slot holding the level-(L-1) masks
    const int stride = p.vs_stride;
    ChunkGrabber grab(&p.lev_grab[p.maxlev + 2 + L], ccnt, nwarps);
    long long c;
    while (grab.next(c, lane)) {
        const Chunk ch = load_chunk(&p.ichunks[ics + c]);
        const int w = ch.v;
        const long long a0 = ch.a0;
        const int na = ch.na;
        int vnext = lane < na ? p.rcol[a0 + lane] : 0;
        uint64_t F[W];
#pragma unroll
        for (int k = 0; k < W; ++k) F[k] = p.hm[(size_t)ch.e * W + k] & s_act[k];
        double sw[PL], aw[PL], cw[PL];
#pragma unroll
        for (int ii = 0; ii < PL; ++ii) {
            sw[ii] = p.sigma[(size_t)w * S + lane + 32 * ii];
            aw[ii] = p.acc[(size_t)w * S + lane + 32 * ii];
        }
#pragma unroll
        for (int ii = 0; ii < PL; ++ii)
            cw[ii] = mask_bit<W>(F, lane + 32 * ii) ? (1.0 + sw[ii] * aw[ii]) / sw[ii] : 0.0;
        for (int base = 0; base < na; base += 32) {
            const bool valid = base + lane < na;
            const int v = vnext;
            vnext = base + 32 + lane < na ? p.rcol[a0 + base + 32 + lane] : 0;
            uint64_t tm[W];
            bool any = false;
            if (valid) {
                const uint64_t *row = p.vs + (size_t)v * stride;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    tm[k] = F[k] & row[par * W + k];
                    any |= tm[k] != 0ull;
                }
                st.arcs += 1;
            } else {
#pragma unroll
                for (int k = 0; k < W; ++k) tm[k] = 0ull;
            }
            unsigned bal = __ballot_sync(kFull, any);
            while (bal) {
                const int i0 = __ffs(bal) - 1;
                bal &= bal - 1;
                const int i1 = bal ? __ffs(bal) - 1 : -1;
                if (bal) bal &= bal - 1;
                const int j1 = i1 < 0 ? i0 : i1;
                const int v0 = __shfl_sync(kFull, v, i0);
                const int v1 = __shfl_sync(kFull, v, j1);
                uint64_t n0[W], n1[W];
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    n0[k] = __shfl_sync(kFull, tm[k], i0);
                    n1[k] = i1 < 0 ? 0ull : __shfl_sync(kFull, tm[k], j1);
                }
                double *r0 = p.acc + (size_t)v0 * S;
                double *r1 = p.acc + (size_t)v1 * S;
#pragma unroll
                for (int ii = 0; ii < PL; ++ii) {
                    const int s = lane + 32 * ii;
                    if (mask_bit<W>(n0, s)) atomicAdd(&r0[s], cw[ii]);
                    if (mask_bit<W>(n1, s)) atomicAdd(&r1[s], cw[ii]);
                }
            }
        }
    }
}

// The rest of a backward step at level L, one thread per entry: delta_s(r_q)
// for the query vertices among the level-L entries (their accumulators are
// complete), and, when the pass goes on, the parity slot shared by levels L
// and L - 2: the level-L bits leave it and the level-(L - 2) bits enter it
// (the push from L - 1 reads them in the next step).
template <int W>
__device__ void level_outputs(const TravParams &p, int L, bool swap, bool set_next, const uint64_t *s_act,
                              const uint64_t *s_need, long long gthr, long long nthr) {
    constexpr int S = 64 * W;
    const int stride = p.vs_stride;
    const int slot = 1 + (L & 1);
    const long long e0 = p.lev_start[L], e1 = e0 + (long long)p.lev_cnt[L];
    for (long long e = e0 + gthr; e < e1; e += nthr) {
        const int v = p.hv[e];
        uint64_t F[W];
#pragma unroll
        for (int k = 0; k < W; ++k) F[k] = p.hm[(size_t)e * W + k];
        if (swap) {
            uint64_t *row = p.vs + (size_t)v * stride;
#pragma unroll
            for (int k = 0; k < W; ++k) atomicAnd((unsigned long long *)&row[slot * W + k], ~(unsigned long long)F[k]);
        }
        const uint64_t qm = p.qmask[v];
        if (!qm) continue;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            uint64_t b = F[k] & s_act[k];
            while (b) {
                const int s = 64 * k + __ffsll((long long)b) - 1;
                b &= b - 1;
                uint64_t x = qm & s_need[s];
                if (!x) continue;
                const double d = p.sigma[(size_t)v * S + s] * p.acc[(size_t)v * S + s];
                while (x) {
                    const int q = __ffsll((long long)x) - 1;
                    x &= x - 1;
                    p.dep[s * 64 + q] = d;
                }
            }
        }
    }
    if (!set_next) return;
    const long long g0 = p.lev_start[L - 2], g1 = g0 + (long long)p.lev_cnt[L - 2];
    for (long long e = g0 + gthr; e < g1; e += nthr) {
        uint64_t *row = p.vs + (size_t)p.hv[e] * stride;
#pragma unroll
        for (int k = 0; k < W; ++k)
            atomicOr((unsigned long long *)&row[slot * W + k], (unsigned long long)p.hm[e * W + k]);
    }
}

// Dependencies on one query vertex r by a vertex scan, from the pair
// dependencies of Eq. 2: r lies on sigma_sr * sigma_rt of the sigma_st
// shortest s-t paths when d(s, r) + d(r, t) = d(s, t) (and on none
// otherwise), so delta_s.(r) = sigma_sr * sum of sigma_rt / sigma_st over
// those t != s, r. rlev and rsig hold d(r, t) and sigma_rt from a forward
// traversal rooted at r. A level-L entry (t, F) lists the sources s with
// d(s, t) = L, so source s takes t exactly when d(s, r) = L - d(r, t), and
// every (t, s) pair is met once, in any order: there is no level order and
// no barrier. Lanes first screen 32 entries at a time on d(r, t) against the
// levels at which the tile's sources meet r; the survivors are taken two at
// a time, each lane adding the terms of its sources l + 32 i in registers.
// Each warp's sums, times sigma_sr, go to vsum with one fp64 atomic add per
// source.
template <int W>
__device__ void vertex_scan(const TravParams &p, int Lmax, const uint64_t *s_need, long long gwarp,
                            long long nwarps) {
    constexpr int S = 64 * W;
    constexpr int PL = 2 * W;
    const int lane = threadIdx.x & 31;
    int ks[PL];  // d(s, r) of the lane's sources, -1 for slots without a query
    double a[PL];
    int kmin = 0x7fffffff, kmax = -1;
    uint64_t kset = 0ull;  // the levels below 64 at which some source meets r
#pragma unroll
    for (int ii = 0; ii < PL; ++ii) {
        const int s = lane + 32 * ii;
        const uint64_t x = s_need[s];
        ks[ii] = x ? p.qlevel[s * 64 + __ffsll((long long)x) - 1] : -1;
        a[ii] = 0.0;
        if (ks[ii] >= 1) {
            kmin = min(kmin, ks[ii]);
            kmax = max(kmax, ks[ii]);
            if (ks[ii] < 64) kset |= 1ull << ks[ii];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
        kset |= __shfl_xor_sync(kFull, kset, o);
    }
    unsigned pairs = 0;
    if (kmax >= 1) {
        for (int L = kmin + 1; L <= Lmax; ++L) {
            const long long eend = p.lev_start[L + 1];
            for (long long b = p.lev_start[L] + 32 * gwarp; b < eend; b += 32 * nwarps) {
                const long long e = b + lane;
                int t = 0, k = -1;
                if (e < eend) {
                    t = p.hv[e];
                    const int dr = p.rlev[t];
                    if (dr >= 1) k = L - dr;
                }
                const bool keep = k >= kmin && k <= kmax && (k >= 64 || ((kset >> k) & 1ull));
                const double rs = keep ? p.rsig[t] : 0.0;
                unsigned bal = __ballot_sync(kFull, keep);
                while (bal) {
                    const int i0 = __ffs(bal) - 1;
                    bal &= bal - 1;
                    const int i1 = bal ? __ffs(bal) - 1 : -1;
                    if (bal) bal &= bal - 1;
                    const int j1 = i1 < 0 ? i0 : i1;
                    const int t0 = __shfl_sync(kFull, t, i0);
                    const int t1 = __shfl_sync(kFull, t, j1);
                    const int k0 = __shfl_sync(kFull, k, i0);
                    const int k1 = i1 < 0 ? -2 : __shfl_sync(kFull, k, j1);  // -2 matches no source
                    const double r0 = __shfl_sync(kFull, rs, i0);
                    const double r1 = __shfl_sync(kFull, rs, j1);
                    uint64_t f0[W], f1[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        f0[w] = p.hm[(b + i0) * W + w];
                        f1[w] = p.hm[(b + j1) * W + w];
                    }
                    const double *q0 = p.sigma + (size_t)t0 * S;
                    const double *q1 = p.sigma + (size_t)t1 * S;
#pragma unroll
                    for (int ii = 0; ii < PL; ++ii) {
                        const int s = lane + 32 * ii;
                        if (ks[ii] == k0 && mask_bit<W>(f0, s)) {
                            a[ii] += r0 / q0[s];
                            ++pairs;
                        }
                        if (ks[ii] == k1 && mask_bit<W>(f1, s)) {
                            a[ii] += r1 / q1[s];
                            ++pairs;
                        }
                    }
                }
            }
        }
    }
    const double *sr = p.sigma + (size_t)p.vroot * S;
#pragma unroll
    for (int ii = 0; ii < PL; ++ii)
        if (a[ii] != 0.0) atomicAdd(&p.vsum[lane + 32 * ii], sr[lane + 32 * ii] * a[ii]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
    if (lane == 0 && pairs) atomicAdd(&p.ctr->vpairs, (unsigned long long)pairs);
}

// Dependencies on several query vertices at once by the vertex scan: the
// form of vertex_scan for a group whose queries sit at up to 64 distinct
// vertices (columns c, vertex croot[c]). rlevq / rsigq [t * 64 + c] hold
// d(croot[c], t) and sigma_{croot[c] t} from one traversal rooted at all the
// columns. Columns go 8 at a time (one 32-byte sector of a row of rlevq).
// Each warp screens 32 level-L entries at a time: entry (t, F) is kept for
// column c when L - d(r_c, t) is a level at which a source of the tile that
// needs c meets r_c (the same screen as the one-vertex scan). For a kept
// (entry, column), each lane adds sigma_{r_c t} / sigma_st, for its sources s
// in F that need c and have d(s, r_c) = L - d(r_c, t), into the block's
// shared sums [s][c]; at the end of the 8 columns the block multiplies them by
// sigma_s(r_c) and adds them into msum [s * 64 + c] with one fp64 atomic each.
// No level order and no grid barrier inside.
template <int W>
__device__ __noinline__ void vertex_scan_multi(const TravParams &p, int Lmax, const uint64_t *s_need, long long gwarp,
                                               long long nwarps) {
    constexpr int S = 64 * W;
    constexpr int PL = 2 * W;
    constexpr int G = W >= 8 ? 4 : 8;  // columns per pass (the shared sums of 512 sources x 8 columns would pass 48 KB)
    __shared__ double s_acc[S * G];
    __shared__ int32_t s_ql[S * G];  // d(s, r_c) for sources that need column c, else -1
    __shared__ int32_t s_kmin[G], s_kmax[G];
    __shared__ unsigned long long s_kset[G];
    const int lane = threadIdx.x & 31;
    unsigned pairs = 0;
    for (int cg = 0; cg < p.ncols; cg += G) {
        const int nc = min(G, p.ncols - cg);
        __syncthreads();
        for (int i = threadIdx.x; i < S * G; i += blockDim.x) {
            s_acc[i] = 0.0;
            s_ql[i] = -1;
        }
        if (threadIdx.x < G) {
            s_kmin[threadIdx.x] = 0x7fffffff;
            s_kmax[threadIdx.x] = -1;
            s_kset[threadIdx.x] = 0ull;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            uint64_t x = s_need[s];
            while (x) {
                const int q = __ffsll((long long)x) - 1;
                x &= x - 1;
                const int j = p.qcol[q] - cg;
                if (j < 0 || j >= nc) continue;
                const int lv = p.qlevel[s * 64 + q];
                if (lv < 1) continue;
                s_ql[s * G + j] = lv;
                atomicMin(&s_kmin[j], lv);
                atomicMax(&s_kmax[j], lv);
                if (lv < 64) atomicOr(&s_kset[j], 1ull << lv);
            }
        }
        __syncthreads();
        int kmin[G], kmax[G];
        unsigned long long kset[G];
        int lfrom = 0x7fffffff;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            kmin[j] = s_kmin[j];
            kmax[j] = s_kmax[j];
            kset[j] = s_kset[j];
            if (kmax[j] >= 1) lfrom = min(lfrom, kmin[j] + 1);
        }
        for (int L = lfrom; L <= Lmax; ++L) {
            const long long eend = p.lev_start[L + 1];
            for (long long b = p.lev_start[L] + 32 * gwarp; b < eend; b += 32 * nwarps) {
                const long long e = b + lane;
                int t = 0;
                unsigned kq = 0;
                int dr[G];
#pragma unroll
                for (int j = 0; j < G; ++j) dr[j] = -1;
                if (e < eend) {
                    t = p.hv[e];
                    const int4 *row = reinterpret_cast<const int4 *>(p.rlevq + (size_t)t * 64 + cg);
#pragma unroll
                    for (int h = 0; h < G / 4; ++h) {
                        const int4 a = row[h];
                        dr[4 * h] = a.x;
                        dr[4 * h + 1] = a.y;
                        dr[4 * h + 2] = a.z;
                        dr[4 * h + 3] = a.w;
                    }
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const int k = L - dr[j];
                        if (j < nc && dr[j] >= 1 && k >= kmin[j] && k <= kmax[j] && (k >= 64 || ((kset[j] >> k) & 1ull)))
                            kq |= 1u << j;
                    }
                }
                unsigned bal = __ballot_sync(kFull, kq != 0u);
                while (bal) {
                    const int i = __ffs(bal) - 1;
                    bal &= bal - 1;
                    const int ti = __shfl_sync(kFull, t, i);
                    unsigned kqi = __shfl_sync(kFull, kq, i);
                    int dri[G];
#pragma unroll
                    for (int j = 0; j < G; ++j) dri[j] = __shfl_sync(kFull, dr[j], i);
                    uint64_t F[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) F[w] = p.hm[(b + i) * W + w];
                    const double *qs = p.sigma + (size_t)ti * S;
                    while (kqi) {
                        const int j = __ffs(kqi) - 1;
                        kqi &= kqi - 1;
                        int drj = 0;
#pragma unroll
                        for (int jj = 0; jj < G; ++jj)
                            if (jj == j) drj = dri[jj];
                        const int k = L - drj;
                        const double rs = p.rsigq[(size_t)ti * 64 + cg + j];
#pragma unroll
                        for (int ii = 0; ii < PL; ++ii) {
                            const int s = lane + 32 * ii;
                            if (mask_bit<W>(F, s) && s_ql[s * G + j] == k) {
                                atomicAdd(&s_acc[s * G + j], rs / qs[s]);
                                ++pairs;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // sigma_s(r_c) times the sums: delta_s.(r_c) parts of this block
        for (int i = threadIdx.x; i < S * G; i += blockDim.x) {
            const double a = s_acc[i];
            if (a != 0.0) {
                const int sl = i / G, j = i % G;
                atomicAdd(&p.msum[sl * 64 + cg + j], a * p.sigma[(size_t)p.croot[cg + j] * S + sl]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
    if (lane == 0 && pairs) atomicAdd(&p.ctr->vpairs, (unsigned long long)pairs);
}

template <int W, int MODE, int MINB>
__global__ void __launch_bounds__(512, MINB) trav_kernel(TravParams p) {
    constexpr int S = 64 * W;
    const int lane = threadIdx.x & 31;
    const long long wpb = blockDim.x >> 5;
    const long long gwarp = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * wpb;
    const long long gthr = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    uint32_t gen = 0;
    __shared__ uint64_t s_need[S];
    __shared__ int32_t s_minql[S];
    __shared__ uint64_t s_active[W];
    __shared__ uint64_t s_active_next[W];
    __shared__ uint64_t s_valid[W];  // the tile's occupied source slots
    __shared__ int32_t s_lstop;
    Stats st;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_mark = timer ? global_ns() : 0ull;
    unsigned long long ns_fwd = 0, ns_bwd = 0, ns_other = 0;

    for (long long tile = 0; tile < p.ntiles; ++tile) {
        const int32_t *tsrc = p.srcs + tile * S;
        check_cancel(p);
        if (blockIdx.x == 0) init_tile<W, MODE>(p, tsrc);
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const int32_t v = tsrc[s];
            s_need[s] = (MODE != kModeReach && v >= 0) ? p.need[v] : 0ull;
        }
        if (threadIdx.x < W) {
            uint64_t m = 0;
            for (int b = 0; b < 64; ++b)
                if (tsrc[threadIdx.x * 64 + b] >= 0) m |= 1ull << b;
            s_valid[threadIdx.x] = m;
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
        }

        // ---------------- forward ----------------
        long long es = 0, cs = 0, ics = 0, es_prev = 0;
        int L = 0;
        long long total = 0;
        for (;;) {
            // the level's entries and chunks, counted in one word by warp_append
            const unsigned long long pk = ld_vol(&p.lev_grab[4 * ((long long)p.maxlev + 2) + L]);
            const long long ecnt = (long long)(pk & 0xffffffffull);
            const long long ccnt = (long long)(pk >> 32);
            const long long iccnt = (long long)ld_vol(&p.lev_grab[2 * ((long long)p.maxlev + 2) + L]);
            const long long es1 = es + ecnt, cs1 = cs + ccnt, ics1 = ics + iccnt;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                p.lev_cnt[L] = (unsigned long long)ecnt;  // published for the passes after the forward
                p.lev_ccnt[L] = (unsigned long long)ccnt;
                p.lev_start[L] = es;
                p.lev_cstart[L] = cs;
                p.lev_start[L + 1] = es1;
                p.lev_cstart[L + 1] = cs1;
                p.lev_icstart[L] = ics;
                p.lev_icstart[L + 1] = ics1;
            }
            if (L >= 1) {
                const int nxt = 1 + ((L + 1) & 1);
                for (long long e = es_prev + gthr; e < es; e += nthr) {
                    const int v = p.hv[e];
                    uint64_t *row = p.vs + (size_t)v * p.vs_stride;
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        atomicAnd((unsigned long long *)&row[nxt * W + w], ~(unsigned long long)p.hm[e * W + w]);
                }
            }
            // direction of level L: bottom-up when its frontier's out-arcs
            // reach the threshold (the same counter in every block)
            const bool pull = MODE != kModeReach && L >= 1 && p.pull_arcs_min > 0 &&
                              (long long)ld_vol(&p.lev_grab[3 * ((long long)p.maxlev + 2) + L]) >= p.pull_arcs_min;
            if (pull) {
                pull_level<W, MODE>(p, L, es, es1, cs1, ics1, st, s_need, s_valid, gwarp, nwarps);
                if (timer) atomicAdd(&p.ctr->pull_levels, 1ull);
            } else {
                forward_level<W, MODE, MINB == 1>(p, L, cs, ccnt, es1, cs1, ics1, st, s_need, gwarp, nwarps);
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            total = es1;
            if ((ld_vol(&p.lev_grab[4 * ((long long)p.maxlev + 2) + L + 1]) & 0xffffffffull) == 0ull) break;
            if (L + 2 > p.maxlev) {
                if (threadIdx.x == 0) set_err(p.ctr, kDevLevelOverflow);
                return;
            }
            es_prev = es;
            es = es1;
            cs = cs1;
            ics = ics1;
            ++L;
        }
        const int Lmax = L;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_fwd += t - t_mark;
            t_mark = t;
            atomicMax(&p.ctr->levels_max, (unsigned long long)Lmax);
        }

        // ---------------- backward ----------------
        if (MODE == kModeScan && (p.flags & kFlagRootOut)) {
            // the query vertices' own traversal (source slot c = column c):
            // keep d(r_c, t) and sigma_{r_c t}
            for (int Lr = 0; Lr <= Lmax; ++Lr) {
                const long long eend = p.lev_start[Lr + 1];
                for (long long e = p.lev_start[Lr] + gthr; e < eend; e += nthr) {
                    const int v = p.hv[e];
                    if (p.ncols >= 2) {
                        uint64_t x = p.hm[(size_t)e * W];  // columns sit in the first mask word
                        while (x) {
                            const int c = __ffsll((long long)x) - 1;
                            x &= x - 1;
                            p.rlevq[(size_t)v * 64 + c] = Lr;
                            p.rsigq[(size_t)v * 64 + c] = p.sigma[(size_t)v * S + c];
                        }
                    } else {
                        p.rlev[v] = Lr;
                        p.rsig[v] = p.sigma[(size_t)v * S];
                    }
                }
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        } else if (MODE == kModeScan && !(p.flags & kFlagNoBackward)) {
            if (p.ncols >= 2)
                vertex_scan_multi<W>(p, Lmax, s_need, gwarp, nwarps);
            else
                vertex_scan<W>(p, Lmax, s_need, gwarp, nwarps);
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        }
        if (MODE == kModeSpd && !(p.flags & kFlagNoBackward)) {
            if (threadIdx.x == 0) s_lstop = 0x7fffffff;
            __syncthreads();
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                int mq = 0x7fffffff;
                if (tsrc[s] >= 0) {
                    if (p.flags & kFlagFullBackward) {
                        mq = 0;
                    } else {
                        uint64_t x = s_need[s];
                        while (x) {
                            const int q = __ffsll((long long)x) - 1;
                            x &= x - 1;
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
            if (lstop <= Lmax) {
                // the parity slot of level Lmax - 1 is empty after the forward pass
                if (Lmax - 1 >= lstop) {
                    const int slot = 1 + ((Lmax - 1) & 1);
                    const long long g0 = p.lev_start[Lmax - 1], g1 = g0 + (long long)p.lev_cnt[Lmax - 1];
                    for (long long e = g0 + gthr; e < g1; e += nthr) {
                        uint64_t *row = p.vs + (size_t)p.hv[e] * p.vs_stride;
#pragma unroll
                        for (int w = 0; w < W; ++w)
                            atomicOr((unsigned long long *)&row[slot * W + w], (unsigned long long)p.hm[e * W + w]);
                    }
                    if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
                }
                for (int Lb = Lmax; Lb >= lstop; --Lb) {
                    if (threadIdx.x < W) {
                        uint64_t a = 0, an = 0;
                        for (int b = 0; b < 64; ++b) {
                            const int mq = s_minql[threadIdx.x * 64 + b];
                            if (mq <= Lb) a |= 1ull << b;
                            if (mq <= Lb - 1) an |= 1ull << b;
                        }
                        s_active[threadIdx.x] = a;
                        s_active_next[threadIdx.x] = an;
                    }
                    __syncthreads();
                    const bool more = Lb > lstop;
                    level_outputs<W>(p, Lb, more, more && Lb - 2 >= lstop, s_active, s_need, gthr, nthr);
                    if (more) {
                        const long long ics = p.lev_icstart[Lb];
                        const long long ic = (long long)ld_vol(&p.lev_grab[2 * ((long long)p.maxlev + 2) + Lb]);
                        push_level<W>(p, Lb, ics, ic, s_active_next, nwarps, st);
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

        if (MODE != kModeReach) flush_stats(p.ctr, st, lane);

        // ---------------- tile end ----------------
        if (MODE == kModeScan && blockIdx.x == 0) {
            // one sum per source (one query vertex) or per (source, column)
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                uint64_t x = s_need[s];
                const double d = p.vsum[s];
                while (x) {
                    const int q = __ffsll((long long)x) - 1;
                    x &= x - 1;
                    p.dep[s * 64 + q] = p.ncols >= 2 ? p.msum[s * 64 + p.qcol[q]] : d;
                }
            }
            __syncthreads();
        }
        if (MODE != kModeReach && blockIdx.x == 0) tile_query_sums(p, tile, S, tsrc, s_need);
        if (MODE == kModeReach) {
            for (long long e = gthr; e < total; e += nthr)
                atomicOr((unsigned long long *)&p.rvmask[p.hv[e]], (unsigned long long)p.hm[e * W]);
        }
        if (!(p.flags & kFlagNoReset)) {
            for (long long e = gwarp; e < total; e += nwarps) {
                const int v = p.hv[e];
                if (MODE != kModeReach) {
                    uint64_t F[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) F[w] = p.hm[e * W + w];
                    double *row = p.sigma + (size_t)v * S;
                    double *arow = p.acc + (size_t)v * S;
#pragma unroll
                    for (int ii = 0; ii < 2 * W; ++ii) {
                        const int s = lane + 32 * ii;
                        if (mask_bit<W>(F, s)) {
                            row[s] = 0.0;
                            if (MODE == kModeSpd) arow[s] = 0.0;
                        }
                    }
                }
                if (lane < p.vs_stride) p.vs[(size_t)v * p.vs_stride + lane] = 0ull;
                if (lane == 0) p.tag[v] = -1;
            }
            if (blockIdx.x == 0) {
                for (int l = threadIdx.x; l <= Lmax + 1; l += blockDim.x) {
                    p.lev_cnt[l] = 0ull;
                    p.lev_ccnt[l] = 0ull;
                    p.lev_grab[l] = 0ull;
                    p.lev_grab[p.maxlev + 2 + l] = 0ull;
                    p.lev_grab[2 * (p.maxlev + 2) + l] = 0ull;
                    p.lev_grab[3 * (p.maxlev + 2) + l] = 0ull;
                    p.lev_grab[4 * (p.maxlev + 2) + l] = 0ull;
                }
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

template <int W, int MODE, int MINB>
bc_status launch(bc_graph *g, TravParams &p) {
    auto kern = trav_kernel<W, MODE, MINB>;
    const int threads = g->block_threads;
    if (threads < 64 * W) return set_error(BC_E_INVALID_ARG, "block_threads must be at least 64 * tile_words");
    const size_t smem = 0;
    int per_sm = 0;
    BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return set_error(BC_E_INTERNAL, "traversal kernel cannot be resident");
    dim3 grid((unsigned)(g->num_sms * per_sm)), block((unsigned)threads);
    void *args[] = {(void *)&p};
    BCD_CUDA(cudaLaunchCooperativeKernel((const void *)kern, grid, block, args, smem, g->stream));
    g->launches += 1;
    g->last_grid = (int)grid.x;
    return BC_OK;
}

}  // namespace

bc_status reset_dense_state(bc_graph *g) {
    bcd_workspace &ws = g->ws;
    if (!ws.vs) return BC_OK;  // no workspace (never built, or freed after a failure)
    BCD_CUDA(cudaMemsetAsync(ws.vs, 0, sizeof(uint64_t) * (size_t)ws.n * ws.vs_stride, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.tag, 0xff, sizeof(int32_t) * (size_t)ws.n, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.sigma, 0, sizeof(double) * (size_t)ws.n * 64 * ws.W, g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.lev_cnt, 0, sizeof(unsigned long long) * (size_t)(ws.maxlev + 2), g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.lev_ccnt, 0, sizeof(unsigned long long) * (size_t)(ws.maxlev + 2), g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.lev_grab, 0, sizeof(unsigned long long) * 6 * (size_t)(ws.maxlev + 2), g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.pdone, 0, sizeof(int32_t) * (size_t)(g->weighted ? ws.pcap : 1), g->stream));
    BCD_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(double) * (g->weighted ? (size_t)1 : (size_t)ws.n * 64 * ws.W), g->stream));
    if (ws.dist) {
        BCD_CUDA(cudaMemsetAsync(ws.dist, 0xff, sizeof(uint64_t) * (size_t)ws.n * 64 * ws.W, g->stream));
        BCD_CUDA(cudaMemsetAsync(ws.bcount, 0, sizeof(unsigned long long) * 2 * (size_t)ws.ring, g->stream));
    }
    return BC_OK;
}

bc_status run_traversal(bc_graph *g, int W, TravParams &p, int *levels_out, unsigned long long *edges_out) {
    for (int attempt = 0; attempt < 6; ++attempt) {
        bcd_workspace &ws = g->ws;
        p.vs = ws.vs;
        p.vs_stride = ws.vs_stride;
        p.tag = ws.tag;
        p.sigma = ws.sigma;
        p.acc = ws.acc;
        p.roff = g->d_roff;  // R(G): in-arcs for the backward push and the weighted sigma pull
        p.rcol = g->d_rcol;
        p.hv = ws.hv;
        p.hm = ws.hm;
        p.hcap = p.mode == kModeReach ? ws.hmcap : ws.hcap;
        p.chunks = ws.chunks;
        p.ichunks = ws.ichunks;
        p.ccap = ws.ccap;
        p.partial = ws.partial;
        p.pdone = ws.pdone;
        p.pcap = ws.pcap;
        p.lev_cnt = ws.lev_cnt;
        p.lev_ccnt = ws.lev_ccnt;
        p.lev_grab = ws.lev_grab;
        p.lev_start = ws.lev_start;
        p.lev_cstart = ws.lev_cstart;
        p.lev_icstart = ws.lev_icstart;
        p.maxlev = ws.maxlev;
        p.ctr = ws.ctr;
        p.n = g->n;
        p.chunk_arcs = g->chunk_arcs;
        p.timeout_ns = g->timeout_ns;
        p.cancel = g->cancel_d;
        p.pull_arcs_min = 0;
        if (!g->weighted && p.mode != kModeReach && g->pull_permille > 0) {
            BCD_TRY(ensure_pull_chunks(g));
            p.pchunks = ws.pchunks;
            p.npchunks = ws.npchunks;
            p.pull_arcs_min = std::max<int64_t>(1, (int64_t)((double)g->m * g->pull_permille / 1000.0));
        }
        BCD_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), g->stream));
        bc_status st = BC_E_INTERNAL;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        const bool timed = cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess;
        if (timed) cudaEventRecord(ev0, g->stream);
        if (p.mode == kModeReach) {
            if (W != 1) return set_error(BC_E_INTERNAL, "reach traversal runs with one mask word");
            st = launch<1, kModeReach, 2>(g, p);
        } else if (g->weighted) {
            p.wt = g->d_w;
            p.roff = g->d_roff;
            p.rcol = g->d_rcol;
            p.rwt = g->d_rw;
            if (W < 1 || W > 16 || (W & (W - 1)) || W > ws.W || ((uint64_t)g->n << 6) * (uint64_t)W > (1ull << 32))
                return set_error(BC_E_INVALID_ARG, "weighted tiles: 1, 2, 4, 8 or 16 words, n * 64 * words <= 2^32");
            p.dist = ws.dist;
            p.hs = ws.hs;
            p.buckets = ws.buckets;
            p.bcount = ws.bcount;
            p.bcap = ws.bcap;
            p.ring = ws.ring;
            p.nw = W;
            p.wshort = g->wshort;
            p.lev_dist = ws.lev_dist;
            st = launch_weighted(g, p);
        } else if (p.mode == kModeScan) {
            if (W == 1)
                st = launch<1, kModeScan, 2>(g, p);
            else if (W == 2)
                st = g->blocks_per_sm == 3 ? launch<2, kModeScan, 3>(g, p) : launch<2, kModeScan, 2>(g, p);
            else if (W == 4)
                st = g->blocks_per_sm == 2 ? launch<4, kModeScan, 2>(g, p) : launch<4, kModeScan, 1>(g, p);
            else if (W == 8)
                st = launch<8, kModeScan, 1>(g, p);
            else
                return set_error(BC_E_INVALID_ARG, "tile words must be 1, 2, 4 or 8");
        } else if (W == 1) {
            st = launch<1, kModeSpd, 2>(g, p);
        } else if (W == 2) {
            st = g->blocks_per_sm == 3 ? launch<2, kModeSpd, 3>(g, p) : launch<2, kModeSpd, 2>(g, p);
        } else if (W == 4) {
            st = g->blocks_per_sm == 2 ? launch<4, kModeSpd, 2>(g, p) : launch<4, kModeSpd, 1>(g, p);
        } else if (W == 8) {
            st = launch<8, kModeSpd, 1>(g, p);
        } else {
            return set_error(BC_E_INVALID_ARG, "tile words must be 1, 2, 4 or 8");
        }
        if (timed) cudaEventRecord(ev1, g->stream);
        if (st != BC_OK) {
            if (timed) {
                cudaEventDestroy(ev0);
                cudaEventDestroy(ev1);
            }
            return st;
        }
        Counters c;
        BCD_CUDA(cudaMemcpyAsync(&c, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, g->stream));
        BCD_CUDA(cudaStreamSynchronize(g->stream));
        g->last_ms_launch = 0;
        if (timed) {
            cudaEventElapsedTime(&g->last_ms_launch, ev0, ev1);
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
        }
        if (c.err == kDevOk) {
            g->last = c;
            if (levels_out) *levels_out = (int)c.levels_max;
            if (edges_out) *edges_out = c.edges;
            g->last_ns_fwd = c.ns_fwd;
            g->last_ns_bwd = c.ns_bwd;
            g->last_ns_other = c.ns_other;
            return BC_OK;
        }
        if (c.err == kDevTimeout) {
            reset_dense_state(g);
            return set_error(BC_E_TIMEOUT, "traversal: a grid barrier wait timed out");
        }
        if (c.err == kDevCancelled) {
            reset_dense_state(g);
            return set_error(BC_E_CANCELLED, "traversal: cancelled by bc_cancel");
        }
        if (c.err == kDevBucketOverflow) {
            // more pending pairs at one distance than a ring slot holds: grow and rerun
            BCD_TRY(grow_buckets(g));
            BCD_TRY(reset_dense_state(g));
            if (p.qflags) BCD_CUDA(cudaMemsetAsync(p.qflags, 0, sizeof(uint32_t) * 64, g->stream));
            continue;
        }
        if (c.err == kDevLevelOverflow) {
            // more non-empty levels than the arrays hold (integer weights): grow and rerun
            BCD_TRY(grow_levels(g));
            BCD_TRY(reset_dense_state(g));
            if (p.qflags) BCD_CUDA(cudaMemsetAsync(p.qflags, 0, sizeof(uint32_t) * 64, g->stream));
            continue;
        }
        // capacity overflow: grow the level history and retry from a clean state
        BCD_TRY(grow_history(g));
        BCD_TRY(reset_dense_state(g));
        if (p.mode == kModeReach && p.rvmask)
            BCD_CUDA(cudaMemsetAsync(p.rvmask, 0, sizeof(uint64_t) * (size_t)g->n, g->stream));
        if (p.qflags) BCD_CUDA(cudaMemsetAsync(p.qflags, 0, sizeof(uint32_t) * 64, g->stream));
    }
    return set_error(BC_E_OOM, "traversal: level history did not fit after growing it");
}

}  // namespace bcd
